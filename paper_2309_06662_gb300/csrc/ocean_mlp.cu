// ocean_mlp.cu -- the learned column closure's network on the tensor cores: BF16 GEMMs
// on tcgen05 with FP32 accumulators in TMEM and fused epilogues (bias, SiLU, SiLU backward, transposed
// copies for the weight gradients), the closure loss and its gradient, Adam on FP32
// master weights, and the trainer handle of the C ABI.
//
// Network (see include/ocean.h): x (6 nz) -> H -> H -> H -> y (3 nz), SiLU after each
// hidden layer.  Layer weights W [in][out]; the GEMMs read W^T [out][in] in the forward
// pass and W [in][out] in the backward pass, both kept as BF16 copies of the FP32 master.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ocean.h"
#include "ocean_internal.cuh"

using bf16 = __nv_bfloat16;

namespace {

// ------------------------------------------------------------------ GEMM (tensor cores)

__device__ __forceinline__ void cp16(void* smem, const void* gmem, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = pred ? 16 : 0;   // src-size 0: the 16 bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// SiLU and its derivative with the fast exponential and division (the results are
// rounded to BF16): for z below about -88, exp(-z) overflows to infinity and the fast
// division returns 0, the limit of both
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.f + __expf(-z)); }
// the forward pass's SiLU with one special-function instruction instead of two:
// z sigmoid(z) = z (1/2 + tanh(z/2) / 2), tanh by the hardware approximation (relative
// error about 2^-11, below the BF16 rounding the result gets)
__device__ __forceinline__ float silu_bf16(float z) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    return z * fmaf(0.5f, t, 0.5f);
}
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = __fdividef(1.f, 1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

enum EpiMode { EPI_F32 = 0, EPI_SILU = 1, EPI_SILU_BWD = 2 };

struct Epi {
    int mode;
    const float* bias;   // [N] (forward modes)
    float* outF;         // fp32 [M][ldF]: C (+bias), or the pre-activation z
    int ldF;
    bf16* outB;          // bf16 [M][ldB]: silu(z), or dz
    int ldB;
    bf16* outT;          // bf16 [N][ldT]: transposed copy of outB (nullable)
    int ldT;
    const float* Zin;    // fp32 [M][ldZ] pre-activation (SiLU backward)
    int ldZ;
};

__device__ __forceinline__ void epi_store(const Epi& e, int m, int n, float acc) {
    if (e.mode == EPI_F32) {
        e.outF[(long)m * e.ldF + n] = acc + (e.bias ? e.bias[n] : 0.f);
    } else if (e.mode == EPI_SILU) {
        const float z = acc + e.bias[n];
        if (e.outF) e.outF[(long)m * e.ldF + n] = z;
        const bf16 h = __float2bfloat16_rn(silu_f(z));
        e.outB[(long)m * e.ldB + n] = h;
        if (e.outT) e.outT[(long)n * e.ldT + m] = h;
    } else {
        const bf16 d = __float2bfloat16_rn(acc * silu_grad_f(e.Zin[(long)m * e.ldZ + n]));
        e.outB[(long)m * e.ldB + n] = d;
        if (e.outT) e.outT[(long)n * e.ldT + m] = d;
    }
}

// ------------------------------------------------------------------ GEMM on tcgen05
//
// C[m][n] = sum_k A[m][k] B[n][k] on Blackwell's fifth-generation tensor cores: one CTA of
// 128 threads per 128 x 128 output tile; K in steps of 64 (one 128-byte swizzle atom of
// BF16), each step staged by cp.async into shared memory in the 128-byte-swizzled
// K-major layout the MMA descriptors describe, double-buffered; one thread issues four
// tcgen05.mma (M 128, N 128, K 16, BF16 in, FP32 accumulate) per step into a 128-column
// TMEM accumulator and commits them to the step's mbarrier, which frees the buffer for
// the load two steps later; the four warps then read their 32 accumulator lanes with
// tcgen05.ld and run the epilogue.  Waits are bounded: a barrier that does not complete
// within ~1 s sets g_tc_err and the tile is abandoned (TMEM is still freed).

constexpr int TBM = 128, TBN = 128, TBK = 64, TTH = 128;
constexpr unsigned TMEM_COLS = 128;
constexpr int TILE_BYTES = TBM * TBK * 2;                        // 16 KB per operand tile
constexpr size_t TC_SMEM = 1024 + 4 * (size_t)TILE_BYTES + 64;  // alignment slack, 2 x (A, B), barriers

__device__ int g_tc_err = 0;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// K-major operand descriptor, 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes
// apart (stride byte offset), leading byte offset unused (1), descriptor version 1
__device__ __forceinline__ unsigned long long sw128_desc(unsigned saddr) {
    unsigned long long d = (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= 1ull << 16;
    d |= (unsigned long long)(1024 >> 4) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N = 128, M = 128
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TBN >> 3) << 17) |
                              ((unsigned)(TBM >> 4) << 24);

// spin on the barrier's phase `parity` for at most `limit` SM clock cycles (~1 s by
// default); false if it did not complete
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          long long limit = 2000000000LL) {
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Epilogue of 32 consecutive columns n0 .. n0+31 of row m held by one thread: the row-major
// outputs go out as 16-byte vectors when the whole run is inside the matrix (the leading
// dimensions are multiples of 8, so the vectors are aligned); the transposed copy is
// written element by element (the lanes of a warp hold consecutive rows, so those
// stores coalesce across the warp).
__device__ __forceinline__ void epi_run32(const Epi& e, int m, int n0, int N, const unsigned* r) {
    if (n0 + 32 > N) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (n0 + j < N) epi_store(e, m, n0 + j, __uint_as_float(r[j]));
        return;
    }
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
    if (e.mode == EPI_SILU_BWD) {
        const float4* z4 = reinterpret_cast<const float4*>(e.Zin + (long)m * e.ldZ + n0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 z = z4[q];
            v[4 * q] *= silu_grad_f(z.x);
            v[4 * q + 1] *= silu_grad_f(z.y);
            v[4 * q + 2] *= silu_grad_f(z.z);
            v[4 * q + 3] *= silu_grad_f(z.w);
        }
    } else if (e.bias) {
        const float4* b4 = reinterpret_cast<const float4*>(e.bias + n0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 bq = b4[q];
            v[4 * q] += bq.x;
            v[4 * q + 1] += bq.y;
            v[4 * q + 2] += bq.z;
            v[4 * q + 3] += bq.w;
        }
    }
    if (e.mode == EPI_F32 || (e.mode == EPI_SILU && e.outF)) {
        float4* o4 = reinterpret_cast<float4*>(e.outF + (long)m * e.ldF + n0);
#pragma unroll
        for (int q = 0; q < 8; ++q) o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (e.mode == EPI_F32) return;
    if (e.mode == EPI_SILU) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = silu_f(v[j]);
    }
    unsigned pk[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        pk[j] = *reinterpret_cast<const unsigned*>(&h2);
    }
    uint4* b4 = reinterpret_cast<uint4*>(e.outB + (long)m * e.ldB + n0);
#pragma unroll
    for (int q = 0; q < 4; ++q) b4[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    if (e.outT) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const unsigned w = pk[j >> 1];
            const unsigned short h = (j & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xFFFFu);
            reinterpret_cast<unsigned short*>(e.outT)[(long)(n0 + j) * e.ldT + m] = h;
        }
    }
}

__global__ void __launch_bounds__(TTH) k_gemm_nt_tc(const bf16* __restrict__ A, int lda,
                                                    const bf16* __restrict__ B, int ldb, int M,
                                                    int N, int K, Epi e) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        ((unsigned long long)tc_raw + 1023) & ~1023ull);
    // buffer b of A at base + b TILE_BYTES, of B at base + (2 + b) TILE_BYTES
    auto sA = [&](int b) { return base + b * TILE_BYTES; };
    auto sB = [&](int b) { return base + (2 + b) * TILE_BYTES; };
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(base + 4 * TILE_BYTES);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bar + 2);
    int* abandon = reinterpret_cast<int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abandon = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;

    // one K step: 128 rows x 8 chunks of 16 bytes per operand, chunk c of row r at
    // r * 128 + ((c ^ (r % 8)) * 16) (the 128-byte swizzle)
    auto load = [&](int kt, int buf) {
        const int k0 = kt * TBK;
        for (int q = tid; q < TBM * 8; q += TTH) {
            const int r = q >> 3, c = q & 7;
            const int gk = k0 + c * 8;
            const unsigned off = (unsigned)(r * 128 + ((c ^ (r & 7)) << 4));
            const int gm = m0 + r, gn = n0 + r;
            const bool pa = gm < M && gk < K, pb = gn < N && gk < K;
            cp16(sA(buf) + off, pa ? (const void*)(A + (long)gm * lda + gk) : (const void*)A, pa);
            cp16(sB(buf) + off, pb ? (const void*)(B + (long)gn * ldb + gk) : (const void*)B, pb);
        }
        cp_commit();
    };
    const int nk = (K + TBK - 1) / TBK;
    unsigned ph = 0u;   // bit b: parity of the next completion of bar[b]
    bool ok = true;
    load(0, 0);
    for (int kt = 0; kt < nk && ok; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            const int nb2 = (kt + 1) & 1;
            if (kt + 1 >= 2) {   // the MMAs of step kt - 1 read that buffer
                ok = __syncthreads_and(mbar_wait(smem_u32(&bar[nb2]), (ph >> nb2) & 1u) ? 1 : 0) != 0;
                ph ^= 1u << nb2;
                if (!ok) break;
            }
            load(kt + 1, nb2);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned long long ad = sw128_desc(smem_u32(sA(buf)));
            const unsigned long long bd = sw128_desc(smem_u32(sB(buf)));
#pragma unroll
            for (int k = 0; k < TBK / 16; ++k) {
                const unsigned acc = (kt > 0 || k > 0) ? 1u : 0u;
                // advancing K by 16 BF16 (32 bytes) inside the swizzle atom: +2 in the
                // 16-byte address field
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad + 2ull * k), "l"(bd + 2ull * k), "r"(TC_IDESC), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&bar[buf]))
                : "memory");
        }
    }
    if (ok) {   // the last commit covers every MMA of this tile
        const int lb = (nk - 1) & 1;
        ok = __syncthreads_and(mbar_wait(smem_u32(&bar[lb]), (ph >> lb) & 1u) ? 1 : 0) != 0;
    }
    if (!ok) {
        atomicExch(&g_tc_err, 1);
        *abandon = 1;
    }
    cp_wait<0>();
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!*abandon) {
        const int row = warp * 32 + lane, m = m0 + row;
#pragma unroll 1
        for (int c0 = 0; c0 < TBN; c0 += 32) {
            unsigned r[32];
            tmem_ld32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, r);
            if (m < M) epi_run32(e, m, n0 + c0, N, r);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(TMEM_COLS));
}

// ------------------------------------------------------------------ GEMM: TMA-fed tcgen05
//
// The same 128 x 128 tile and MMA sequence as k_gemm_nt_tc, with the operands brought in
// by the tensor memory accelerator: one thread issues, per K step of 64, a 2-D bulk tensor
// copy of the A tile (128 rows) and of the B tile (128 rows), 128-byte swizzled, into a
// ring of GS stages; a second thread issues the MMAs of a stage once its full barrier
// has counted the copied bytes and commits them to the stage's empty barrier, which the
// copying thread waits for before reusing the stage; the last commit signals the
// epilogue.  Rows and K beyond the matrix arrive as zeros (the copies' out-of-bounds
// fill).  Needs the rows of A and B 16-byte aligned (leading dimensions multiples of 8).
// Eight warps read the accumulator: warp w the lanes 32 (w % 4).. and the column half
// w / 4, so the epilogue runs on twice the warps of the loading scheme.

constexpr int GS = 2, TMA_TH = 256;
constexpr size_t TMA_SMEM = 1024 + 2 * GS * (size_t)TILE_BYTES + 128;

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__global__ void __launch_bounds__(TMA_TH) k_gemm_nt_tma(const __grid_constant__ CUtensorMap tA,
                                                     const __grid_constant__ CUtensorMap tB,
                                                     int M, int N, int K, Epi e) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        ((unsigned long long)tc_raw + 1023) & ~1023ull);
    auto sA = [&](int st) { return base + st * TILE_BYTES; };
    auto sB = [&](int st) { return base + (GS + st) * TILE_BYTES; };
    unsigned long long* full = reinterpret_cast<unsigned long long*>(base + 2 * GS * TILE_BYTES);
    unsigned long long* empty = full + GS;
    unsigned long long* done = empty + GS;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(done + 1);
    int* abandon = reinterpret_cast<int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int nk = (K + TBK - 1) / TBK;

    if (tid == 0) {
        for (int st = 0; st < GS; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[st])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abandon = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- copies: stage kt % GS, after the MMAs of step kt - GS released it
        int issued = 0;
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % GS, use = kt / GS;
            if (kt >= GS && !mbar_wait(smem_u32(&empty[st]), (unsigned)(use - 1) & 1u)) {
                atomicExch(&g_tc_err, 1);
                *abandon = 1;
                break;
            }
            mbar_expect(smem_u32(&full[st]), 2u * TILE_BYTES);
            tma_load_2d(smem_u32(sA(st)), &tA, kt * TBK, m0, smem_u32(&full[st]));
            tma_load_2d(smem_u32(sB(st)), &tB, kt * TBK, n0, smem_u32(&full[st]));
            ++issued;
        }
        // on an abandoned tile, wait (bounded) for the copies still in flight
        if (*abandon)
            for (int kt = (issued > GS ? issued - GS : 0); kt < issued; ++kt)
                mbar_wait(smem_u32(&full[kt % GS]), (unsigned)(kt / GS) & 1u);
    } else if (warp == 1 && lane == 0) {
        // ---- MMAs: four K-16 steps per stage into the TMEM accumulator
        for (int kt = 0; kt < nk; ++kt) {
            const int st = kt % GS, use = kt / GS;
            if (!mbar_wait(smem_u32(&full[st]), (unsigned)use & 1u)) {
                atomicExch(&g_tc_err, 1);
                *abandon = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const unsigned long long ad = sw128_desc(smem_u32(sA(st)));
            const unsigned long long bd = sw128_desc(smem_u32(sB(st)));
#pragma unroll
            for (int k = 0; k < TBK / 16; ++k) {
                const unsigned acc = (kt > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad + 2ull * k), "l"(bd + 2ull * k), "r"(TC_IDESC), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&empty[st]))
                : "memory");
        }
        // arrives once every MMA issued above has completed
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(done))
            : "memory");
    }
    const bool ok = __syncthreads_and(mbar_wait(smem_u32(done), 0u) ? 1 : 0) != 0;
    if (!ok) {
        atomicExch(&g_tc_err, 1);
        *abandon = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!*abandon) {
        // the tile's bias in shared memory (the operand stages are free once `done` has
        // completed): every row reads the same 128 values
        Epi ee = e;
        if (e.bias && e.mode != EPI_SILU_BWD) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            float* sb = reinterpret_cast<float*>(base);
            for (int q = tid; q < TBN; q += TMA_TH) sb[q] = n0 + q < N ? e.bias[n0 + q] : 0.f;
            __syncthreads();
            ee.bias = sb - n0;   // indexed by the matrix column n0 + c
        }
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane, m = m0 + row;
        if (e.mode == EPI_SILU && !e.outF && !e.outT && e.bias) {
            // the network's hidden layers: SiLU in BF16 through a shared-memory tile, so
            // that the rows leave as whole 256-byte segments (one thread per row would
            // write 32 rows per store instruction); rows padded by 16 bytes
            constexpr int LDT = TBN * 2 + 16;
            unsigned char* tile = base + 1024;
#pragma unroll 1
            for (int c0 = half * (TBN / 2); c0 < (half + 1) * (TBN / 2); c0 += 32) {
                unsigned r[32];
                tmem_ld32(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)c0, r);
                unsigned pk[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + 2 * j;
                    const float b0 = n < N ? ee.bias[n] : 0.f, b1 = n + 1 < N ? ee.bias[n + 1] : 0.f;
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(
                        silu_bf16(__uint_as_float(r[2 * j]) + b0), silu_bf16(__uint_as_float(r[2 * j + 1]) + b1));
                    pk[j] = *reinterpret_cast<const unsigned*>(&h2);
                }
                uint4* dst = reinterpret_cast<uint4*>(tile + row * LDT + c0 * 2);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
            __syncthreads();
            // 16 chunks of 16 bytes per row; the leading dimension and N are multiples of 8
            for (int q = tid; q < TBM * (TBN / 8); q += TMA_TH) {
                const int rr = q / (TBN / 8), cc = (q % (TBN / 8)) * 8;
                if (m0 + rr < M && n0 + cc < N)
                    *reinterpret_cast<uint4*>(e.outB + (long)(m0 + rr) * e.ldB + n0 + cc) =
                        *reinterpret_cast<const uint4*>(tile + rr * LDT + cc * 2);
            }
        } else {
#pragma unroll 1
            for (int c0 = half * (TBN / 2); c0 < (half + 1) * (TBN / 2); c0 += 32) {
                unsigned r[32];
                tmem_ld32(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)c0, r);
                if (m < M) epi_run32(ee, m, n0 + c0, N, r);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(TMEM_COLS));
}

// tensor map of a row-major BF16 matrix [rows][ld] read K columns wide, boxes of 64
// columns x TBM rows, 128-byte swizzle; false if the driver refuses it
bool gemm_tensor_map(CUtensorMap* map, const bf16* ptr, int rows, int K, int ld) {
    const unsigned long long dims[2] = {(unsigned long long)K, (unsigned long long)rows};
    const unsigned long long strides[1] = {(unsigned long long)ld * sizeof(bf16)};
    const unsigned box[2] = {(unsigned)TBK, (unsigned)TBM};
    return oc_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box,
                           CU_TENSOR_MAP_SWIZZLE_128B);
}

// Self-test of the bounded wait: a barrier that nothing completes; the wait gives up
// after `limit` cycles and the kernel reports it instead of hanging
__global__ void k_wait_selftest(long long limit, int* timed_out) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(smem_u32(&bar), 0u, limit);
    if (threadIdx.x == 0) *timed_out = ok ? 0 : 1;
}

// ------------------------------------------------------------------ GEMM: persistent tcgen05
//
// The network's forward pass (bias + SiLU to BF16, or bias to FP32) as a persistent,
// warp-specialised kernel: each block walks the 128 x 128 output tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; warp 0 issues the tensor copies of every K step into a
// ring of PGS stages, warp 1 issues the MMAs into one of two TMEM accumulators (128
// columns each), and warps 2..9 drain an accumulator (each its 32 TMEM lanes and one
// column half) while the MMAs of the next tile fill the other.  Barriers: full/empty per
// stage (copies landed / MMAs done with the stage), accf/acce per accumulator (MMAs of a
// tile done / its eight epilogue warps have read it).  The hidden layers' BF16 rows go out through a
// warp-private shared-memory tile as whole 256-byte row segments.  Every wait is bounded;
// after one gives up, all later waits of the block return at once and the block exits
// (the closure's error status is set).

// eight epilogue warps: two per TMEM lane quarter, each draining one column half
// five operand stages (one block per SM): enough copies in flight to keep the MMAs fed
constexpr int PGS = 5, PG_EW = 8, PG_TH = (2 + PG_EW) * 32, PG_LDT = TBN + 16;
constexpr size_t PG_STAGE = PG_EW * 32 * (size_t)PG_LDT;          // per warp 32 rows x 64 columns
constexpr size_t PG_SMEM = 1024 + 2 * PGS * (size_t)TILE_BYTES + PG_STAGE + 256 * 4 + 256;

__device__ __forceinline__ bool pg_wait(unsigned bar, unsigned parity, volatile int* abandon) {
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abandon) return false;
        if (clock64() - t0 > 2000000000LL) {
            *abandon = 1;
            atomicExch(&g_tc_err, 1);
            return false;
        }
    }
}

__global__ void __launch_bounds__(PG_TH) k_gemm_nt_pers(const __grid_constant__ CUtensorMap tA,
                                                      const __grid_constant__ CUtensorMap tB,
                                                      int M, int N, int K, Epi e) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        ((unsigned long long)tc_raw + 1023) & ~1023ull);
    auto sA = [&](int st) { return base + st * TILE_BYTES; };
    auto sB = [&](int st) { return base + (PGS + st) * TILE_BYTES; };
    unsigned char* stage = base + 2 * PGS * TILE_BYTES;
    float* sbias = reinterpret_cast<float*>(stage + PG_STAGE);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sbias + 256);
    unsigned long long* empty = full + PGS;
    unsigned long long* accf = empty + PGS;
    unsigned long long* acce = accf + 2;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(acce + 2);
    volatile int* abandon = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntn = (N + TBN - 1) / TBN, ntiles = ((M + TBM - 1) / TBM) * ntn;
    const int nk = (K + TBK - 1) / TBK;

    for (int q = tid; q < 256; q += PG_TH) sbias[q] = (e.bias && q < N) ? e.bias[q] : 0.f;
    if (tid == 0) {
        for (int st = 0; st < PGS; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[st])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acce[b])),
                         "r"((unsigned)PG_EW));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abandon = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(2u * TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {   // ---- copies
            int g = 0;
            for (int t = blockIdx.x; t < ntiles && !*abandon; t += gridDim.x) {
                const int m0 = (t / ntn) * TBM, n0 = (t % ntn) * TBN;
                for (int kt = 0; kt < nk; ++kt, ++g) {
                    const int st = g % PGS, use = g / PGS;
                    if (g >= PGS && !pg_wait(smem_u32(&empty[st]), (unsigned)(use - 1) & 1u, abandon))
                        break;
                    mbar_expect(smem_u32(&full[st]), 2u * TILE_BYTES);
                    tma_load_2d(smem_u32(sA(st)), &tA, kt * TBK, m0, smem_u32(&full[st]));
                    tma_load_2d(smem_u32(sB(st)), &tB, kt * TBK, n0, smem_u32(&full[st]));
                }
            }
            // copies still in flight when the block gave up: wait (bounded) for them
            if (*abandon)
                for (int gg = (g > PGS ? g - PGS : 0); gg < g; ++gg) {
                    const long long t0 = clock64();
                    unsigned ok = 0;
                    while (!ok && clock64() - t0 < 2000000000LL)
                        asm volatile(
                            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                            " selp.u32 %0, 1, 0, p;\n}\n"
                            : "=r"(ok)
                            : "r"(smem_u32(&full[gg % PGS])), "r"((unsigned)(gg / PGS) & 1u)
                            : "memory");
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---- MMAs
            int g = 0, i = 0;
            for (int t = blockIdx.x; t < ntiles && !*abandon; t += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !pg_wait(smem_u32(&acce[b]), (unsigned)((i >> 1) - 1) & 1u, abandon))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const unsigned acc_addr = tmem + (unsigned)(b * (int)TMEM_COLS);
                bool fine = true;
                for (int kt = 0; kt < nk; ++kt, ++g) {
                    const int st = g % PGS;
                    if (!pg_wait(smem_u32(&full[st]), (unsigned)(g / PGS) & 1u, abandon)) {
                        fine = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const unsigned long long ad = sw128_desc(smem_u32(sA(st)));
                    const unsigned long long bd = sw128_desc(smem_u32(sB(st)));
#pragma unroll
                    for (int k = 0; k < TBK / 16; ++k) {
                        const unsigned acc = (kt > 0 || k > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_addr),
                            "l"(ad + 2ull * k), "l"(bd + 2ull * k), "r"(TC_IDESC), "r"(acc));
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                            smem_u32(&empty[st]))
                        : "memory");
                }
                if (!fine) break;
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                        smem_u32(&accf[b]))
                    : "memory");
            }
        }
    } else {   // ---- epilogue: warps 2..9, the TMEM lanes 32 (warp % 4) .., column half
        const int quarter = warp & 3, row = quarter * 32 + lane, ch = ((warp - 2) / 4) * (TBN / 2);
        unsigned char* mine = stage + (size_t)(warp - 2) * 32 * PG_LDT;   // this warp's rows
        const bool silu = e.mode == EPI_SILU;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int b = i & 1, m0 = (t / ntn) * TBM, n0 = (t % ntn) * TBN, m = m0 + row;
            if (!pg_wait(smem_u32(&accf[b]), (unsigned)(i >> 1) & 1u, abandon)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
            for (int c0 = ch; c0 < ch + TBN / 2; c0 += 32) {
                unsigned r[32];
                tmem_ld32(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(b * (int)TMEM_COLS + c0), r);
                if (silu) {
                    unsigned pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + c0 + 2 * j;
                        const float z0 = __uint_as_float(r[2 * j]) + (n < N ? sbias[n] : 0.f);
                        const float z1 = __uint_as_float(r[2 * j + 1]) + (n + 1 < N ? sbias[n + 1] : 0.f);
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(silu_bf16(z0), silu_bf16(z1));
                        pk[j] = *reinterpret_cast<const unsigned*>(&h2);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(mine + lane * PG_LDT + (c0 - ch) * 2);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                } else if (m < M) {
                    if (n0 + c0 + 32 <= N) {   // ldF is a multiple of 4: 16-byte vectors
                        float4* o4 = reinterpret_cast<float4*>(e.outF + (long)m * e.ldF + n0 + c0);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int n = n0 + c0 + 4 * q;
                            o4[q] = make_float4(__uint_as_float(r[4 * q]) + sbias[n],
                                                __uint_as_float(r[4 * q + 1]) + sbias[n + 1],
                                                __uint_as_float(r[4 * q + 2]) + sbias[n + 2],
                                                __uint_as_float(r[4 * q + 3]) + sbias[n + 3]);
                        }
                    } else {
                        for (int j = 0; j < 32; ++j) {
                            const int n = n0 + c0 + j;
                            if (n < N) e.outF[(long)m * e.ldF + n] = __uint_as_float(r[j]) + sbias[n];
                        }
                    }
                }
            }
            // the accumulator is read: the MMAs of tile i + 2 may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&acce[b]))
                             : "memory");
            if (silu) {   // this warp's 32 half rows out as 128-byte segments, four per store
                for (int q = lane; q < 32 * (TBN / 16); q += 32) {
                    const int rr = q / (TBN / 16), cc = (q % (TBN / 16)) * 8;
                    if (m0 + quarter * 32 + rr < M && n0 + ch + cc < N)
                        *reinterpret_cast<uint4*>(e.outB + (long)(m0 + quarter * 32 + rr) * e.ldB + n0 + ch + cc) =
                            *reinterpret_cast<const uint4*>(mine + rr * PG_LDT + cc * 2);
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(2u * TMEM_COLS));
}

// A [M][lda], B [N][ldb] row-major BF16 (lda, ldb and K multiples of 8, 16-byte aligned
// rows): TMA-fed when the driver encodes both tensor maps, else staged by cp.async
void gemm_nt(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const Epi& e,
             cudaStream_t s) {
    const dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
    CUtensorMap ta, tb;
    if (gemm_tensor_map(&ta, A, M, K, lda) && gemm_tensor_map(&tb, B, N, K, ldb))
        k_gemm_nt_tma<<<grid, TMA_TH, TMA_SMEM, s>>>(ta, tb, M, N, K, e);
    else
        k_gemm_nt_tc<<<grid, TTH, TC_SMEM, s>>>(A, lda, B, ldb, M, N, K, e);
}

// the network's forward GEMMs (bias + SiLU to BF16 rows, or bias to FP32 rows): the
// persistent kernel, one block per SM, when both tensor maps encode and N <= 256, else
// gemm_nt
void gemm_nt_forward(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K,
                     const Epi& e, cudaStream_t s) {
    const bool plain = (e.mode == EPI_SILU && e.outB && !e.outF && !e.outT) ||
                       (e.mode == EPI_F32 && e.outF && (e.ldF % 4) == 0);
    CUtensorMap ta, tb;
    if (plain && N <= 256 && gemm_tensor_map(&ta, A, M, K, lda) &&
        gemm_tensor_map(&tb, B, N, K, ldb)) {
        const int tiles = ((M + TBM - 1) / TBM) * ((N + TBN - 1) / TBN);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int grid = tiles < sms ? tiles : sms;
        k_gemm_nt_pers<<<grid, PG_TH, PG_SMEM, s>>>(ta, tb, M, N, K, e);
        return;
    }
    gemm_nt(A, lda, B, ldb, M, N, K, e, s);
}

// ------------------------------------------------------------------ fused forward pass
//
// The whole network on one 128-column tile without leaving the SM: the hidden activations
// stay in shared memory, written by the epilogue in the 128-byte-swizzled K-major layout
// the next layer's MMAs read as their A operand, so HBM sees only the features in and the
// outputs out (the four separate GEMMs move every hidden layer through HBM twice).
// Roles, per tile and layer (use u = 4 n + l of the block's n-th tile):
// - warp 0 streams per tile and layer the weight K-blocks (64 inputs x up to 256 outputs,
//   BF16, from L2: the same weights serve every tile) through a ring of FM_S stages;
// - warp 18 streams the tiles' feature K-blocks (128 columns x 64 features) from HBM
//   through a ring of their own (FM_SX stages), so that the next tile's features load
//   while this tile's later layers run;
// - warp 1 issues the MMAs (M 128, N the layer's width, K 16) into TMEM accumulator u mod 2
//   (two of 256 columns: the next layer's sums build up while the epilogue still drains
//   this one);
// - warps 2..17 drain the accumulator (two TMEM loads of 32 columns per warp), release
//   it once both are in registers, and write bias + SiLU as BF16 into the activation tile,
//   each K-block announced on its own barrier: the next layer's MMAs start on K-blocks 0
//   and 1 while the others are still being written.  The last layer's bias-added sums
//   go to FP32 rows of Y.
// Barriers: full/empty per weight stage, fullx/emptyx per feature stage; accf[b] (the MMAs of the accumulator's use done);
// acce[b] (its sixteen epilogue warps have read it); actf[kb] (the eight epilogue warps
// that write K-block kb of the next layer's input have written it).  Every wait is bounded as in
// k_gemm_nt_pers.
constexpr int FM_S = 3, FM_SX = 3, FM_EW = 16, FM_TH = (3 + FM_EW) * 32;
constexpr int FM_XW = 2 + FM_EW;                       // the feature-copy warp
constexpr int FM_ACT = 4 * TILE_BYTES;                 // 128 rows x 256 BF16: four K-blocks
constexpr int FM_B = 256 * TBK * 2;                    // up to 256 weight rows x 64 BF16
constexpr int FM_NBAR = 2 * FM_S + 2 * FM_SX + 2 + 2 + 4;   // full, empty, fullx, emptyx, accf, acce, actf
constexpr size_t FM_SMEM = 1024 + FM_ACT + FM_S * (size_t)FM_B + FM_SX * (size_t)TILE_BYTES +
                           4 * 256 * 4 + FM_NBAR * 8 + 16;
static_assert(FM_SMEM <= 227 * 1024, "fused network's shared memory");

struct FusedMaps {
    CUtensorMap X, W[4];   // features [M][K0] (boxes 64 x 128), W_l^T [N_l][K_l] (64 x NB_l)
};
struct FusedArgs {
    const float* bias[4];
    float* Y;
    int ldY, M, K0, H, N4;
};

__device__ __forceinline__ unsigned fm_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(TBM >> 4) << 24);
}

// byte offset of (row r, column c) of a BF16 tile in the 128-byte-swizzled K-major layout
// of K-blocks of 64 columns: 8-row atoms of 1024 bytes, the 16-byte chunk of each row
// rotated by the row within its atom (the layout TMA writes with SWIZZLE_128B)
__device__ __forceinline__ unsigned sw128_offset(int r, int c) {
    const int kb = c >> 6, j = (c & 63) >> 3;
    return (unsigned)(kb * TILE_BYTES + (r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4) +
                      (c & 7) * 2);
}

// 32 columns of this thread's TMEM lane into r, without waiting (tcgen05.wait::ld follows)
__device__ __forceinline__ void tmem_ld32_async(unsigned taddr, unsigned* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// SiLU of eight sums z = acc + b as BF16, in the half-argument form: with h = z / 2,
// SiLU(z) = z (1 + tanh(z / 2)) / 2 = h + h tanh(h); hb holds b / 2, so h = acc / 2 + hb
// is one packed FMA per pair; tanh is the special-function unit's approximation (the
// result is rounded to BF16)
__device__ __forceinline__ uint4 silu8_bf16(const unsigned* r, const float* hb) {
    const float4 b0 = *reinterpret_cast<const float4*>(hb);
    const float4 b1 = *reinterpret_cast<const float4*>(hb + 4);
    const float hbv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    unsigned pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 h = __ffma2_rn(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])),
                                    make_float2(0.5f, 0.5f), make_float2(hbv[2 * j], hbv[2 * j + 1]));
        float2 t;
        asm("tanh.approx.f32 %0, %1;" : "=f"(t.x) : "f"(h.x));
        asm("tanh.approx.f32 %0, %1;" : "=f"(t.y) : "f"(h.y));
        const float2 s = __ffma2_rn(h, t, h);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(s.x, s.y);
        pk[j] = *reinterpret_cast<const unsigned*>(&h2);
    }
    return make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

__global__ void __launch_bounds__(FM_TH, 1) k_mlp_fused(const __grid_constant__ FusedMaps tm,
                                                        FusedArgs a) {
    extern __shared__ unsigned char fm_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        ((unsigned long long)fm_raw + 1023) & ~1023ull);
    unsigned char* act = base;
    auto sB = [&](int st) { return base + FM_ACT + st * FM_B; };                      // weights
    auto sX = [&](int st) { return base + FM_ACT + FM_S * FM_B + st * TILE_BYTES; };  // features
    // [4][256]: b / 2 of the hidden layers (the SiLU's half argument), b of the last
    float* sbias = reinterpret_cast<float*>(base + FM_ACT + FM_S * FM_B + FM_SX * TILE_BYTES);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sbias + 4 * 256);
    unsigned long long* empty = full + FM_S;
    unsigned long long* fullx = empty + FM_S;
    unsigned long long* emptyx = fullx + FM_SX;
    unsigned long long* accf = emptyx + FM_SX;
    unsigned long long* acce = accf + 2;
    unsigned long long* actf = acce + 2;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(actf + 4);
    volatile int* abandon = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // layer shapes: K-blocks of the inputs (K0, then H), MMA widths (H, then N4 rounded up
    // to 16; H is a multiple of 16)
    const int nkb0 = (a.K0 + TBK - 1) / TBK, nact = (a.H + TBK - 1) / TBK;
    const int nb3 = (a.N4 + 15) & ~15;
    auto NB = [&](int l) { return l < 3 ? a.H : nb3; };
    auto nkb = [&](int l) { return l == 0 ? nkb0 : nact; };
    const int ntiles = (a.M + TBM - 1) / TBM;

    for (int q = tid; q < 4 * 256; q += FM_TH) {
        const int l = q >> 8, c = q & 255;
        const float* bp = l == 0 ? a.bias[0] : l == 1 ? a.bias[1] : l == 2 ? a.bias[2] : a.bias[3];
        sbias[q] = c < (l < 3 ? a.H : a.N4) ? (l < 3 ? 0.5f : 1.f) * bp[c] : 0.f;
    }
    // the activation tile's columns at and beyond H are never written: zero them once
    for (int q = tid; q < FM_ACT / 16; q += FM_TH)
        reinterpret_cast<uint4*>(act)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int st = 0; st < FM_S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[st])));
        }
        for (int st = 0; st < FM_SX; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&fullx[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&emptyx[st])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acce[b])),
                         "r"((unsigned)FM_EW));
        }
        for (int kb = 0; kb < 4; ++kb)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&actf[kb])),
                         "r"((unsigned)FM_EW / 2));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abandon = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    // the zeroed activation tile is read by the tensor cores (the async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tmem_slot;

    // copies still in flight when the block gave up: wait (bounded) for them; the g-th
    // copy of a ring of ns stages completes phase g / ns of stage g mod ns
    auto drain = [&](unsigned long long* bars, int ns, int g) {
        for (int gg = (g > ns ? g - ns : 0); gg < g; ++gg) {
            const long long t0 = clock64();
            unsigned ok = 0;
            while (!ok && clock64() - t0 < 2000000000LL)
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(ok)
                    : "r"(smem_u32(&bars[gg % ns])), "r"((unsigned)(gg / ns) & 1u)
                    : "memory");
        }
    };
    if (warp == 0) {
        if (lane == 0) {   // ---- weight copies: per tile and layer its K-blocks
            int g = 0;
            for (int t = blockIdx.x; t < ntiles && !*abandon; t += gridDim.x)
                for (int l = 0; l < 4 && !*abandon; ++l)
                    for (int kb = 0; kb < nkb(l); ++kb, ++g) {
                        const int st = g % FM_S, use = g / FM_S;
                        if (g >= FM_S &&
                            !pg_wait(smem_u32(&empty[st]), (unsigned)(use - 1) & 1u, abandon))
                            break;
                        mbar_expect(smem_u32(&full[st]), (unsigned)NB(l) * TBK * 2);
                        tma_load_2d(smem_u32(sB(st)), &tm.W[l], kb * TBK, 0, smem_u32(&full[st]));
                    }
            if (*abandon) drain(full, FM_S, g);
        }
    } else if (warp == FM_XW) {
        if (lane == 0) {   // ---- feature copies: per tile its K-blocks
            int g = 0;
            for (int t = blockIdx.x; t < ntiles && !*abandon; t += gridDim.x)
                for (int kb = 0; kb < nkb0; ++kb, ++g) {
                    const int st = g % FM_SX, use = g / FM_SX;
                    if (g >= FM_SX &&
                        !pg_wait(smem_u32(&emptyx[st]), (unsigned)(use - 1) & 1u, abandon))
                        break;
                    mbar_expect(smem_u32(&fullx[st]), (unsigned)TILE_BYTES);
                    tma_load_2d(smem_u32(sX(st)), &tm.X, kb * TBK, t * TBM, smem_u32(&fullx[st]));
                }
            if (*abandon) drain(fullx, FM_SX, g);
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ---- MMAs: layer l of the n-th tile is use u = 4 n + l
            int g = 0, gx = 0, u = 0;
            bool fine = true;
            for (int t = blockIdx.x, n = 0; t < ntiles && fine; t += gridDim.x, ++n)
                for (int l = 0; l < 4 && fine; ++l, ++u) {
                    const int b = u & 1;
                    // accumulator b drained by the epilogue of use u - 2
                    if (u >= 2 && !pg_wait(smem_u32(&acce[b]), (unsigned)((u >> 1) - 1) & 1u, abandon)) {
                        fine = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const unsigned idesc = fm_idesc(NB(l));
                    const unsigned dt = tmem + (unsigned)(b * 256);
                    for (int kb = 0; kb < nkb(l); ++kb, ++g) {
                        const int st = g % FM_S;
                        if (!pg_wait(smem_u32(&full[st]), (unsigned)(g / FM_S) & 1u, abandon)) {
                            fine = false;
                            break;
                        }
                        // layer 0: the tile's feature K-block; layers 1..3: K-block kb of
                        // the input, written by the epilogue of layer l - 1 of this tile (the
                        // (3 n + l - 1)-th phase of actf[kb])
                        const int sx = gx % FM_SX;
                        if (l == 0 ? !pg_wait(smem_u32(&fullx[sx]), (unsigned)(gx / FM_SX) & 1u, abandon)
                                   : !pg_wait(smem_u32(&actf[kb]), (unsigned)(3 * n + l - 1) & 1u, abandon)) {
                            fine = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const unsigned long long ad =
                            sw128_desc(smem_u32(l == 0 ? sX(sx) : act + kb * TILE_BYTES));
                        const unsigned long long bd = sw128_desc(smem_u32(sB(st)));
#pragma unroll
                        for (int k = 0; k < TBK / 16; ++k) {
                            const unsigned acc = (kb > 0 || k > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                "l"(ad + 2ull * k), "l"(bd + 2ull * k), "r"(idesc), "r"(acc));
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                smem_u32(&empty[st]))
                            : "memory");
                        if (l == 0) {
                            asm volatile(
                                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                    smem_u32(&emptyx[sx]))
                                : "memory");
                            ++gx;
                        }
                    }
                    if (!fine) break;
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                            smem_u32(&accf[b]))
                        : "memory");
                }
        }
    } else if (warp < FM_XW) {   // ---- epilogue: warps 2..17, TMEM lanes 32 (warp % 4) ..
        // warp group g = (warp - 2) / 4 owns the 32-column chunks g and g + 4: chunk g lies in
        // K-block g / 2 (0 or 1), chunk g + 4 in K-block g / 2 + 2, so the sixteen warps
        // complete K-blocks 0 and 1 first; eight warps write each K-block
        const int quarter = warp & 3, row = quarter * 32 + lane, grp = (warp - 2) >> 2;
        const unsigned lanes = (unsigned)(quarter * 32) << 16;
        const int ch[2] = {grp, grp + 4};
        int u = 0;
        bool fine = true;
        for (int t = blockIdx.x; t < ntiles && fine; t += gridDim.x) {
            const int m = t * TBM + row;
            for (int l = 0; l < 4; ++l, ++u) {
                const int b = u & 1;
                if (!pg_wait(smem_u32(&accf[b]), (unsigned)(u >> 1) & 1u, abandon)) {
                    fine = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const float* bl = sbias + l * 256;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = ch[h] * 32, kb = ch[h] >> 1;
                    const bool valid = c0 < NB(l);
                    unsigned r[32];
                    if (valid) {
                        tmem_ld32_async(tmem + lanes + (unsigned)(b * 256 + c0), r);
                        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    }
                    if (h == 1) {   // both chunks read: accumulator b is free for use u + 2
                        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0)
                            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(
                                             smem_u32(&acce[b]))
                                         : "memory");
                    }
                    if (l < 3) {   // bias + SiLU, BF16, into the activation tile (0 beyond H)
                        if (kb < nact) {
                            if (valid) {
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const int c = c0 + 8 * q;
                                    const uint4 v = c < a.H ? silu8_bf16(&r[8 * q], bl + c)
                                                            : make_uint4(0u, 0u, 0u, 0u);
                                    *reinterpret_cast<uint4*>(act + sw128_offset(row, c)) = v;
                                }
                            }
                            // this warp's part of K-block kb of the next layer's input is in
                            // shared memory, for the tensor cores (the async proxy)
                            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                            __syncwarp();
                            if (lane == 0)
                                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(
                                                 smem_u32(&actf[kb]))
                                             : "memory");
                        }
                    } else if (valid && m < a.M) {   // bias, FP32 rows of Y
                        float* y = a.Y + (long)m * a.ldY;
                        if (c0 + 32 <= a.N4) {   // ldY is a multiple of 4: 16-byte vectors
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 bb = *reinterpret_cast<const float4*>(bl + c0 + 4 * q);
                                reinterpret_cast<float4*>(y + c0)[q] = make_float4(
                                    __uint_as_float(r[4 * q]) + bb.x, __uint_as_float(r[4 * q + 1]) + bb.y,
                                    __uint_as_float(r[4 * q + 2]) + bb.z, __uint_as_float(r[4 * q + 3]) + bb.w);
                            }
                        } else {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj)
                                if (c0 + jj < a.N4) y[c0 + jj] = __uint_as_float(r[jj]) + bl[c0 + jj];
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512u));
}

// tensor map of a row-major BF16 matrix [rows][ld], K columns, boxes of 64 columns x
// box_rows rows, 128-byte swizzle; false if the driver refuses it
bool fused_tensor_map(CUtensorMap* map, const bf16* ptr, int rows, int K, int ld, int box_rows) {
    const unsigned long long dims[2] = {(unsigned long long)K, (unsigned long long)rows};
    const unsigned long long strides[1] = {(unsigned long long)ld * sizeof(bf16)};
    const unsigned box[2] = {(unsigned)TBK, (unsigned)box_rows};
    return oc_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box,
                           CU_TENSOR_MAP_SWIZZLE_128B);
}

// the fused forward pass for M columns, when the shapes allow it (hidden width and output
// width at most 256, multiples of 16 and of 4 for the widths, the FP32 rows of Y 16-byte
// aligned) and the driver encodes the tensor maps; false to fall back to four GEMMs
bool mlp_fused_forward(const bf16* X, int M, const void* const* Wt, const float* const* b,
                       const int* dims, float* Y, cudaStream_t s) {
    const int K0 = dims[0], H = dims[1], N4 = dims[4];
    if (H > 256 || H % 16 || dims[2] != H || dims[3] != H || N4 > 256 || N4 % 4 || K0 % 8 || M < 1)
        return false;
    FusedMaps tm;
    const int nb[4] = {H, H, H, (N4 + 15) & ~15};
    if (!fused_tensor_map(&tm.X, X, M, K0, K0, TBM)) return false;
    for (int l = 0; l < 4; ++l)
        if (!fused_tensor_map(&tm.W[l], reinterpret_cast<const bf16*>(Wt[l]), dims[l + 1], dims[l],
                              dims[l], nb[l]))
            return false;
    FusedArgs fa{{b[0], b[1], b[2], b[3]}, Y, N4, M, K0, H, N4};
    const int tiles = (M + TBM - 1) / TBM;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_mlp_fused<<<tiles < sms ? tiles : sms, FM_TH, FM_SMEM, s>>>(tm, fa);
    return true;
}

// ------------------------------------------------------------------ elementwise kernels

// fp32 [M][C] -> bf16 [M][ldo] (and, if T, bf16 transpose [C][ldt])
__global__ void k_to_bf16(const float* __restrict__ x, int M, int C, bf16* __restrict__ o,
                          int ldo, bf16* __restrict__ t, int ldt) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)M * C) return;
    const int m = (int)(q / C), c = (int)(q % C);
    const bf16 b = __float2bfloat16_rn(x[q]);
    o[(long)m * ldo + c] = b;
    if (t) t[(long)c * ldt + m] = b;
}

// sum over m of dz^T rows: db[o] = sum_m dzT[o][m]
__global__ void k_rowsum(const bf16* __restrict__ dzT, int ld, int M, int N, float* __restrict__ out) {
    const int o = blockIdx.x;
    if (o >= N) return;
    float s = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += __bfloat162float(dzT[(long)o * ld + m]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[o] = red[0];
}

// counts of the face and wet masks of a batch (2 ints)
__global__ void k_count_masks(const unsigned char* __restrict__ face,
                              const unsigned char* __restrict__ wet, long n, int* out) {
    int a = 0, b = 0;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        a += face[q] != 0;
        b += wet[q] != 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], a);
        atomicAdd(&out[1], b);
    }
}

__device__ __forceinline__ float softplus_f(float z) { return z > 20.f ? z : log1pf(__expf(z)); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + __expf(-z)); }

// Closure loss: per column m and level k, with kap = kappa softplus(y_k),
//   rT = (-kap dzT - FT)/sFT, rS likewise on faces; qT = (gT y_{nz+k} - GT)/sGT, qS on
//   wet levels; L = (sum rT^2 + rS^2)/n_face + (sum qT^2 + qS^2)/n_wet.
// Writes dL/dy as bf16 [M][3nz] and its transpose, and per-block partial losses.
__global__ void k_closure_loss(const float* __restrict__ Y, int M, int nz, ocean_closure_scales sc,
                               const float* __restrict__ dzT, const float* __restrict__ dzS,
                               const float* __restrict__ FT, const float* __restrict__ FS,
                               const float* __restrict__ GT, const float* __restrict__ GS,
                               const unsigned char* __restrict__ face,
                               const unsigned char* __restrict__ wet, const int* __restrict__ counts,
                               bf16* __restrict__ dY, bf16* __restrict__ dYt, int ldt,
                               double* __restrict__ partial) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const float nf = fmaxf(1.f, (float)counts[0]), nw = fmaxf(1.f, (float)counts[1]);
    double l = 0.0;
    if (q < (long)M * nz) {
        const int m = (int)(q / nz), k = (int)(q % nz);
        const float* y = Y + (long)m * 3 * nz;
        const float yk = y[k], ykap = sc.kappa * softplus_f(yk);
        float dk = 0.f, dgt = 0.f, dgs = 0.f;
        if (face[q]) {
            const float rT = (-ykap * dzT[q] - FT[q]) / sc.sFT;
            const float rS = (-ykap * dzS[q] - FS[q]) / sc.sFS;
            l += (double)rT * rT + (double)rS * rS;
            l /= nf;
            dk = (2.f * rT * (-dzT[q]) / sc.sFT + 2.f * rS * (-dzS[q]) / sc.sFS) / nf;
            dk *= sc.kappa * sigmoid_f(yk);
        }
        if (wet[q]) {
            const float qT = (sc.gT * y[nz + k] - GT[q]) / sc.sGT;
            const float qS = (sc.gS * y[2 * nz + k] - GS[q]) / sc.sGS;
            l += ((double)qT * qT + (double)qS * qS) / nw;
            dgt = 2.f * qT / sc.sGT * sc.gT / nw;
            dgs = 2.f * qS / sc.sGS * sc.gS / nw;
        }
        const long base = (long)m * 3 * nz;
        const bf16 b0 = __float2bfloat16_rn(dk), b1 = __float2bfloat16_rn(dgt), b2 = __float2bfloat16_rn(dgs);
        dY[base + k] = b0;
        dY[base + nz + k] = b1;
        dY[base + 2 * nz + k] = b2;
        dYt[(long)k * ldt + m] = b0;
        dYt[(long)(nz + k) * ldt + m] = b1;
        dYt[(long)(2 * nz + k) * ldt + m] = b2;
    }
    __shared__ double red[256];
    red[threadIdx.x] = l;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* __restrict__ p, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += p[b];
        out[0] = s;
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights of one layer, then the two BF16
// copies: W [in][out] and W^T [out][in]
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long n, int out, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16* __restrict__ wb, bf16* __restrict__ wt,
                       int in) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    w[q] = wq;
    if (wb) {
        const bf16 b = __float2bfloat16_rn(wq);
        wb[q] = b;
        const int i = (int)(q / out), o = (int)(q % out);
        wt[(long)o * in + i] = b;
    }
}

__global__ void k_weight_copies(const float* __restrict__ w, long n, int out, int in,
                                bf16* __restrict__ wb, bf16* __restrict__ wt) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const bf16 b = __float2bfloat16_rn(w[q]);
    wb[q] = b;
    const int i = (int)(q / out), o = (int)(q % out);
    wt[(long)o * in + i] = b;
}

inline int nb(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// the GEMM's shared memory (above the default 48 KB); called before the first launch on a
// device and outside stream capture
int closure_gemm_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_nt_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TC_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_nt_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TMA_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gemm_nt_pers, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PG_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FM_SMEM);
    return (int)e;
}

// runs k_wait_selftest on `s`; 1 if the wait gave up (the expected outcome), 0 if it
// completed, -1 on a CUDA error
int closure_wait_selftest(long long limit, cudaStream_t s) {
    int* d = nullptr;
    int h = -1;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return -1;
    k_wait_selftest<<<1, 32, 0, s>>>(limit, d);
    if (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        h = -1;
    cudaFree(d);
    return h;
}

// 1 if a closure GEMM abandoned a tile on a barrier that did not complete since the last
// call (the flag is cleared); call after synchronising the stream the GEMMs ran on
int closure_gemm_failed() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(int)) != cudaSuccess) return 1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_err, &z, sizeof(int));
    }
    return v;
}

// ------------------------------------------------------------------ inference inside the step

// y = MLP(x) for M columns of bf16 features Xb [M][dims0], weights W^T (bf16 [out][in])
// and biases per layer, hidden activations ping-ponging through H0/H1 (bf16 [M][H])
void closure_forward(const void* Xb, int M, const void* const* Wt, const float* const* b,
                     const int* dims, void* H0, void* H1, float* Y, cudaStream_t s) {
    const bf16* a = reinterpret_cast<const bf16*>(Xb);
    if (mlp_fused_forward(a, M, Wt, b, dims, Y, s)) return;
    int lda = dims[0];
    bf16* H[2] = {reinterpret_cast<bf16*>(H0), reinterpret_cast<bf16*>(H1)};
    for (int l = 0; l < 4; ++l) {
        Epi e{};
        e.bias = b[l];
        if (l < 3) {
            e.mode = EPI_SILU;
            e.outB = H[l & 1];
            e.ldB = dims[l + 1];
        } else {
            e.mode = EPI_F32;
            e.outF = Y;
            e.ldF = dims[l + 1];
        }
        gemm_nt_forward(a, lda, reinterpret_cast<const bf16*>(Wt[l]), dims[l], M, dims[l + 1], dims[l], e, s);
        if (l < 3) {
            a = H[l & 1];
            lda = dims[l + 1];
        }
    }
}

namespace {
__global__ void k_transpose_bf16(const float* __restrict__ w, long n, int out, int in,
                                 bf16* __restrict__ wt) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = (int)(q / out), o = (int)(q % out);
    wt[(long)o * in + i] = __float2bfloat16_rn(w[q]);
}
}  // namespace

// W^T [out][in] in bf16 from fp32 W [in][out] on the device (the forward pass's operand)
void closure_weight_transpose(const float* W, int in, int out, void* Wt, cudaStream_t s) {
    const long n = (long)in * out;
    k_transpose_bf16<<<nb(n, 256), 256, 0, s>>>(W, n, out, in, reinterpret_cast<bf16*>(Wt));
}

// ------------------------------------------------------------------ trainer handle

struct ocean_mlp_s {
    int nz = 0, hidden = 0, max_batch = 0;
    int dims[5] = {};
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    // per layer
    float *W[4] = {}, *b[4] = {}, *gW[4] = {}, *gb[4] = {}, *mW[4] = {}, *vW[4] = {}, *mb[4] = {},
          *vb[4] = {};
    bf16 *Wb[4] = {}, *Wt[4] = {};
    // activations of one batch
    bf16 *X = nullptr, *Xt = nullptr, *H[3] = {}, *Ht[3] = {}, *dYb = nullptr, *dYt = nullptr,
         *dZ[2] = {}, *dZt[2] = {};
    float *Z[3] = {}, *Y = nullptr;
    double *partial = nullptr, *lossd = nullptr;
    int* counts = nullptr;
    long step = 0;
    std::string err;
};

namespace {

int mfail(ocean_mlp_t h, int code, const char* msg) {
    if (h) h->err = msg;
    oc_set_last_error(msg);
    return code;
}

template <typename T>
T* dalloc(ocean_mlp_t h, size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) return nullptr;
    h->allocs.push_back(p);
    cudaMemsetAsync(p, 0, n * sizeof(T), h->stream);
    return reinterpret_cast<T*>(p);
}

// forward pass of M rows of bf16 features already in h->X; keeps Z, H (and their
// transposes when train) for the backward pass; output fp32 Y [M][out]
void forward(ocean_mlp_t h, int M, bool train, float* Yout) {
    cudaStream_t s = h->stream;
    const bf16* a = h->X;
    int lda = h->dims[0];
    for (int l = 0; l < 4; ++l) {
        const int in = h->dims[l], out = h->dims[l + 1];
        Epi e{};
        if (l < 3) {
            e.mode = EPI_SILU;
            e.bias = h->b[l];
            e.outF = train ? h->Z[l] : nullptr;
            e.ldF = out;
            e.outB = h->H[l];
            e.ldB = out;
            e.outT = train ? h->Ht[l] : nullptr;
            e.ldT = h->max_batch;
        } else {
            e.mode = EPI_F32;
            e.bias = h->b[l];
            e.outF = Yout;
            e.ldF = out;
        }
        gemm_nt(a, lda, h->Wt[l], in, M, out, in, e, s);
        if (l < 3) {
            a = h->H[l];
            lda = out;
        }
    }
}

// gradients of the closure loss for a batch (forward included); loss to host
int loss_and_grads(ocean_mlp_t h, const ocean_batch* bt, int M, const ocean_closure_scales* sc,
                   float* loss) {
    cudaStream_t s = h->stream;
    const int nz = h->nz, in0 = h->dims[0], out = h->dims[4], MB = h->max_batch;
    k_to_bf16<<<nb((long)M * in0, 256), 256, 0, s>>>(bt->X, M, in0, h->X, in0, h->Xt, MB);
    forward(h, M, true, h->Y);
    cudaMemsetAsync(h->counts, 0, 2 * sizeof(int), s);
    k_count_masks<<<64, 256, 0, s>>>(bt->face, bt->wet, (long)M * nz, h->counts);
    const int lb = nb((long)M * nz, 256);
    k_closure_loss<<<lb, 256, 0, s>>>(h->Y, M, nz, *sc, bt->dzT, bt->dzS, bt->FT, bt->FS, bt->GT,
                                      bt->GS, bt->face, bt->wet, h->counts, h->dYb, h->dYt, MB,
                                      h->partial);
    k_sum_partials<<<1, 32, 0, s>>>(h->partial, lb, h->lossd);
    // backward: layer 4 (linear), then 3, 2, 1 (SiLU)
    const bf16* dz = h->dYb;
    const bf16* dzt = h->dYt;
    for (int l = 3; l >= 0; --l) {
        const int li = h->dims[l], lo = h->dims[l + 1];
        const bf16* actT = l > 0 ? h->Ht[l - 1] : h->Xt;   // [li][MB]
        Epi ew{};
        ew.mode = EPI_F32;
        ew.outF = h->gW[l];
        ew.ldF = lo;
        gemm_nt(actT, MB, dzt, MB, li, lo, M, ew, s);       // dW[i][o] = sum_m a[m][i] dz[m][o]
        k_rowsum<<<lo, 256, 0, s>>>(dzt, MB, M, lo, h->gb[l]);
        if (l > 0) {
            const int nxt = l & 1;
            Epi ed{};
            ed.mode = EPI_SILU_BWD;
            ed.outB = h->dZ[nxt];
            ed.ldB = li;
            ed.outT = h->dZt[nxt];
            ed.ldT = MB;
            ed.Zin = h->Z[l - 1];
            ed.ldZ = li;
            gemm_nt(dz, lo, h->Wb[l], lo, M, li, lo, ed, s);   // dh[m][i] = sum_o dz[m][o] W[i][o]
            dz = h->dZ[nxt];
            dzt = h->dZt[nxt];
        }
    }
    (void)out;
    if (loss) {
        double L = 0.0;
        if (cudaMemcpyAsync(&L, h->lossd, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return mfail(h, OCEAN_ERR_CUDA, "loss copy failed");
        *loss = (float)L;
        if (closure_gemm_failed())
            return mfail(h, OCEAN_ERR_TIMEOUT, "a tensor-core GEMM tile timed out on its barrier");
    }
    return cudaGetLastError() == cudaSuccess ? OCEAN_OK : mfail(h, OCEAN_ERR_CUDA, "kernel launch failed");
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

size_t ocean_mlp_param_count(int nz, int hidden) {
    if (nz < 1 || hidden < 16) return 0;
    const size_t d[5] = {(size_t)6 * nz, (size_t)hidden, (size_t)hidden, (size_t)hidden, (size_t)3 * nz};
    size_t n = 0;
    for (int l = 0; l < 4; ++l) n += d[l] * d[l + 1] + d[l + 1];
    return n;
}

int ocean_mlp_create(int nz, int hidden, int max_batch, const float* params, void* stream,
                     ocean_mlp_t* out) {
    if (!out) return mfail(nullptr, OCEAN_ERR_ARG, "null output handle");
    *out = nullptr;
    if (nz < 1 || nz > OC_NZMAX || hidden < 16 || hidden % 16 || max_batch < 1 || max_batch % 8)
        return mfail(nullptr, OCEAN_ERR_ARG,
                     "ocean_mlp_create: need 1 <= nz <= 192, hidden a multiple of 16, max_batch a positive multiple of 8");
    ocean_mlp_t h = new ocean_mlp_s();
    h->nz = nz;
    h->hidden = hidden;
    h->max_batch = max_batch;
    h->stream = (cudaStream_t)stream;
    if (closure_gemm_setup() != (int)cudaSuccess) {
        delete h;
        return mfail(nullptr, OCEAN_ERR_CUDA, "GEMM shared-memory attribute could not be set");
    }
    const int d[5] = {6 * nz, hidden, hidden, hidden, 3 * nz};
    memcpy(h->dims, d, sizeof d);
    bool ok = true;
    for (int l = 0; l < 4 && ok; ++l) {
        const size_t nw = (size_t)d[l] * d[l + 1], nbias = d[l + 1];
        ok = (h->W[l] = dalloc<float>(h, nw)) && (h->b[l] = dalloc<float>(h, nbias)) &&
             (h->gW[l] = dalloc<float>(h, nw)) && (h->gb[l] = dalloc<float>(h, nbias)) &&
             (h->mW[l] = dalloc<float>(h, nw)) && (h->vW[l] = dalloc<float>(h, nw)) &&
             (h->mb[l] = dalloc<float>(h, nbias)) && (h->vb[l] = dalloc<float>(h, nbias)) &&
             (h->Wb[l] = dalloc<bf16>(h, nw)) && (h->Wt[l] = dalloc<bf16>(h, nw));
    }
    const size_t MB = max_batch;
    ok = ok && (h->X = dalloc<bf16>(h, MB * d[0])) && (h->Xt = dalloc<bf16>(h, MB * d[0])) &&
         (h->Y = dalloc<float>(h, MB * d[4])) && (h->dYb = dalloc<bf16>(h, MB * d[4])) &&
         (h->dYt = dalloc<bf16>(h, MB * d[4])) && (h->partial = dalloc<double>(h, MB * nz / 256 + 2)) &&
         (h->lossd = dalloc<double>(h, 1)) && (h->counts = dalloc<int>(h, 2));
    for (int l = 0; l < 3 && ok; ++l)
        ok = (h->H[l] = dalloc<bf16>(h, MB * hidden)) && (h->Ht[l] = dalloc<bf16>(h, MB * hidden)) &&
             (h->Z[l] = dalloc<float>(h, MB * hidden));
    for (int l = 0; l < 2 && ok; ++l)
        ok = (h->dZ[l] = dalloc<bf16>(h, MB * (size_t)hidden)) && (h->dZt[l] = dalloc<bf16>(h, MB * (size_t)hidden));
    if (!ok) {
        ocean_mlp_destroy(h);
        return mfail(nullptr, OCEAN_ERR_OOM, "ocean_mlp_create: device allocation failed");
    }
    if (params) {
        int rc = ocean_mlp_set_params(h, params, ocean_mlp_param_count(nz, hidden));
        if (rc) {
            ocean_mlp_destroy(h);
            return rc;
        }
    }
    *out = h;
    return OCEAN_OK;
}

void ocean_mlp_destroy(ocean_mlp_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    delete h;
}

int ocean_mlp_set_params(ocean_mlp_t h, const float* host, size_t count) {
    if (!h || !host) return mfail(h, OCEAN_ERR_ARG, "null argument");
    if (count != ocean_mlp_param_count(h->nz, h->hidden))
        return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_set_params: wrong parameter count");
    const float* p = host;
    for (int l = 0; l < 4; ++l) {
        const size_t nw = (size_t)h->dims[l] * h->dims[l + 1], nbias = h->dims[l + 1];
        cudaMemcpyAsync(h->W[l], p, nw * sizeof(float), cudaMemcpyHostToDevice, h->stream);
        p += nw;
        cudaMemcpyAsync(h->b[l], p, nbias * sizeof(float), cudaMemcpyHostToDevice, h->stream);
        p += nbias;
        k_weight_copies<<<nb(nw, 256), 256, 0, h->stream>>>(h->W[l], nw, h->dims[l + 1], h->dims[l],
                                                          h->Wb[l], h->Wt[l]);
        cudaMemsetAsync(h->mW[l], 0, nw * sizeof(float), h->stream);
        cudaMemsetAsync(h->vW[l], 0, nw * sizeof(float), h->stream);
        cudaMemsetAsync(h->mb[l], 0, nbias * sizeof(float), h->stream);
        cudaMemsetAsync(h->vb[l], 0, nbias * sizeof(float), h->stream);
    }
    h->step = 0;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return mfail(h, OCEAN_ERR_CUDA, "ocean_mlp_set_params: copy failed");
    return OCEAN_OK;
}

int ocean_mlp_get_params(ocean_mlp_t h, float* host, size_t count) {
    if (!h || !host) return mfail(h, OCEAN_ERR_ARG, "null argument");
    if (count != ocean_mlp_param_count(h->nz, h->hidden))
        return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_get_params: wrong parameter count");
    float* p = host;
    for (int l = 0; l < 4; ++l) {
        const size_t nw = (size_t)h->dims[l] * h->dims[l + 1], nbias = h->dims[l + 1];
        cudaMemcpyAsync(p, h->W[l], nw * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
        p += nw;
        cudaMemcpyAsync(p, h->b[l], nbias * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
        p += nbias;
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return mfail(h, OCEAN_ERR_CUDA, "ocean_mlp_get_params: copy failed");
    return OCEAN_OK;
}

int ocean_selftest_bounded_wait(long long cycles, void* stream) {
    if (cycles < 1) return mfail(nullptr, OCEAN_ERR_ARG, "cycles must be >= 1");
    const int r = closure_wait_selftest(cycles, (cudaStream_t)stream);
    if (r < 0) return mfail(nullptr, OCEAN_ERR_CUDA, "self-test kernel failed");
    if (r == 1) return mfail(nullptr, OCEAN_ERR_TIMEOUT, "bounded wait gave up (self-test: expected)");
    return OCEAN_OK;
}

int ocean_mlp_forward_bf16(ocean_mlp_t h, const void* d_Xb, int M, float* d_Y) {
    if (!h || !d_Xb || !d_Y) return mfail(h, OCEAN_ERR_ARG, "null argument");
    if (M < 1 || M > h->max_batch) return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_forward_bf16: 1 <= M <= max_batch");
    if (((uintptr_t)d_Xb & 15) != 0) return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_forward_bf16: d_Xb must be 16-byte aligned");
    const void* Wt[4] = {h->Wt[0], h->Wt[1], h->Wt[2], h->Wt[3]};
    const float* b[4] = {h->b[0], h->b[1], h->b[2], h->b[3]};
    closure_forward(d_Xb, M, Wt, b, h->dims, h->H[0], h->H[1], d_Y, h->stream);
    return cudaGetLastError() == cudaSuccess ? OCEAN_OK : mfail(h, OCEAN_ERR_CUDA, "kernel launch failed");
}

int ocean_mlp_forward(ocean_mlp_t h, const float* d_X, int M, float* d_Y) {
    if (!h || !d_X || !d_Y) return mfail(h, OCEAN_ERR_ARG, "null argument");
    if (M < 1 || M > h->max_batch) return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_forward: 1 <= M <= max_batch");
    const int in0 = h->dims[0];
    k_to_bf16<<<nb((long)M * in0, 256), 256, 0, h->stream>>>(d_X, M, in0, h->X, in0, nullptr, 0);
    forward(h, M, false, d_Y);
    return cudaGetLastError() == cudaSuccess ? OCEAN_OK : mfail(h, OCEAN_ERR_CUDA, "kernel launch failed");
}

int ocean_mlp_loss_grad(ocean_mlp_t h, const ocean_batch* batch, int M,
                        const ocean_closure_scales* sc, float* loss, float* host_grads) {
    if (!h || !batch || !sc) return mfail(h, OCEAN_ERR_ARG, "null argument");
    if (M < 1 || M > h->max_batch || M % 8)
        return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_loss_grad: M must be a multiple of 8 in [8, max_batch]");
    int rc = loss_and_grads(h, batch, M, sc, loss);
    if (rc) return rc;
    if (host_grads) {
        float* p = host_grads;
        for (int l = 0; l < 4; ++l) {
            const size_t nw = (size_t)h->dims[l] * h->dims[l + 1], nbias = h->dims[l + 1];
            cudaMemcpyAsync(p, h->gW[l], nw * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
            p += nw;
            cudaMemcpyAsync(p, h->gb[l], nbias * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
            p += nbias;
        }
        if (cudaStreamSynchronize(h->stream) != cudaSuccess)
            return mfail(h, OCEAN_ERR_CUDA, "gradient copy failed");
    }
    return OCEAN_OK;
}

int ocean_mlp_train_step(ocean_mlp_t h, const ocean_batch* batch, int M,
                         const ocean_closure_scales* sc, float lr, float* loss) {
    if (!h || !batch || !sc) return mfail(h, OCEAN_ERR_ARG, "null argument");
    if (M < 1 || M > h->max_batch || M % 8)
        return mfail(h, OCEAN_ERR_ARG, "ocean_mlp_train_step: M must be a multiple of 8 in [8, max_batch]");
    int rc = loss_and_grads(h, batch, M, sc, loss);
    if (rc) return rc;
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)h->step), c2 = 1.f - powf(b2, (float)h->step);
    for (int l = 0; l < 4; ++l) {
        const long nw = (long)h->dims[l] * h->dims[l + 1], nbias = h->dims[l + 1];
        k_adam<<<nb(nw, 256), 256, 0, h->stream>>>(h->W[l], h->gW[l], h->mW[l], h->vW[l], nw,
                                                   h->dims[l + 1], lr, b1, b2, eps, c1, c2,
                                                   h->Wb[l], h->Wt[l], h->dims[l]);
        k_adam<<<nb(nbias, 256), 256, 0, h->stream>>>(h->b[l], h->gb[l], h->mb[l], h->vb[l], nbias,
                                                      1, lr, b1, b2, eps, c1, c2, nullptr, nullptr, 1);
    }
    return cudaGetLastError() == cudaSuccess ? OCEAN_OK : mfail(h, OCEAN_ERR_CUDA, "kernel launch failed");
}

}  // extern "C"
