// ocean_kernels.cu -- CUDA kernels of one baroclinic step (sm_103a), instantiated for
// FP64 (R = double) and the mixed form (R = float).
//
// Step n -> n+1 (arXiv 2309.06662, Sec. "New numerical methods ..." and
// Sec. "Optimization of ocean free surface dynamics"):
//   k_diag      hydrostatic pressure (top -> bottom), w from continuity (bottom -> top),
//               Richardson-number kappa and nu: the two intermediates the paper's fused
//               tendency kernels depend on (pressure and vertical diffusivity)
//   k_tracer    WENO-Z flux-form T and S tendencies, quasi-AB2 predictor and the
//               backward-Euler vertical diffusion (Thomas) of the same column, fused;
//               2.5-D tiled (see "tile layout")
//   k_momentum  vector-invariant u and v tendencies (WENO-Z vorticity flux, Coriolis,
//               kinetic-energy and pressure gradients, vertical advection, wind),
//               quasi-AB2, vertical viscosity solve, column sums for the barotropic mode;
//               2.5-D tiled
//   k_baro_*    split-explicit barotropic sub-cycle with equal-weight averaging, BS
//               substeps per pass on shared-memory regions (temporal blocking)
//   k_correct   barotropic correction of u and v
//   k_halo*     periodic halo copies
// One thread owns one water column; threads of a warp hold neighbouring columns of a
// row and walk the same levels, so every level access is coalesced.
#include "ocean_internal.cuh"

namespace {

constexpr int TPB = 128;

// multiplications that the compiler may not fuse into a neighbouring add
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
// reciprocal of a Thomas pivot (>= 1 by construction): exact in FP64, the fast
// approximate reciprocal (2 ulp) in the mixed form
__device__ __forceinline__ double rcp_pivot(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_pivot(float x) { return __fdividef(1.0f, x); }

inline int nblocks(long n, int tpb) { return (int)((n + tpb - 1) / tpb); }

// T and S are stored as anomalies T' = T - Tref(k), S' = S - Sref(k) from horizontally
// uniform reference profiles; in FP32 this keeps ~1e-9 instead of ~1e-6 of absolute
// resolution in the buoyancy that drives the horizontal pressure gradients.
// Buoyancy anomaly b' = g (alpha T' - beta_s S'): its pressure integral differs from the
// full one by a function of k alone, which has no horizontal gradient.
// Explicitly rounded: columns of different depth run this in loops of different trip
// counts, and identical inputs must give identical bits at every level whatever code
// the compiler generates for each trip (the lake-at-rest state depends on it).
template <typename R>
__device__ __forceinline__ R buoy_anom(const KP<R>& p, R Ta, R Sa) {
    return rmul(p.grav, fma(p.alpha, Ta, -rmul(p.beta_s, Sa)));
}

// ------------------------------------------------------------------ diagnostics

// Each kernel body below is a device function of the model's parameters and of the
// position of its work item (a column counter, a tile or a region), called by the
// kernel of one model (position from blockIdx) and by the ensemble's persistent kernels
// (position from a work list), so both run the same code.

// column c of the (nx + 2) x (ny + 2) ring-extended horizontal grid
template <typename R>
__device__ __forceinline__ void diag_col(const KP<R>& p, const long c, const R* __restrict__ u,
                                         const R* __restrict__ v, const R* __restrict__ T,
                                         const R* __restrict__ S, R* __restrict__ w,
                                         R* __restrict__ pr, R* __restrict__ kap,
                                         R* __restrict__ nu) {
    const GeoD& g = p.g;
    const int W = g.nx + 2;
    if (c >= (long)W * (g.ny + 2)) return;
    const int i = (int)(c % W) - 1, j = (int)(c / W) - 1;
    const long c2 = ix2(g, i, j);
    const int kb = g.kb[c2], nz = g.nz;
    if (kb >= nz) return;
    const long P = g.plane;
    // pressure anomaly, integrated downward from the surface (T and S of eight levels
    // loaded at once; the recurrence is serial)
    R bup = buoy_anom(p, T[(nz - 1) * P + c2], S[(nz - 1) * P + c2]);
    R pk = -rmul(bup, p.ptop);
    pr[(nz - 1) * P + c2] = pk;
#pragma unroll 1
    for (int k4 = nz - 2; k4 >= kb; k4 -= 8) {
        R tq[8], sq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool in = k4 - q >= kb;
            tq[q] = in ? T[(long)(k4 - q) * P + c2] : R(0);
            sq[q] = in ? S[(long)(k4 - q) * P + c2] : R(0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k4 - q;
            if (k < kb) break;
            R bk = buoy_anom(p, tq[q], sq[q]);
            pk = fma(-rmul(R(0.5), bk + bup), p.dzf[k + 1], pk);
            pr[k * P + c2] = pk;
            bup = bk;
        }
    }
    // one upward sweep: w on the bottom faces, integrated from the sea floor, and the
    // Richardson-number closure on the interior faces, from the levels k-1 (kept in
    // registers) and k
    const R dy = p.dy, dxvS = p.dxv[j + OC_H], dxvN = p.dxv[j + 1 + OC_H], rac = p.rAc[j + OC_H];
    R wk = R(0);
    w[kb * P + c2] = wk;
    R Tm = R(0), Sm = R(0), ub = R(0), vb = R(0);
    // every lane of the warp walks the same levels (from the warp's deepest sea floor),
    // so that each load instruction reads one level's row: coalesced
    const int kw = __reduce_min_sync(__activemask(), kb);
    for (int k4 = kw; k4 < nz; k4 += 4) {
        R Tq[4], Sq[4], u0q[4], u1q[4], v0q[4], v1q[4];   // four levels' operands at once
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long ck = (long)(k4 + q) * P + c2;
            const bool in = k4 + q < nz && k4 + q >= kb;
            Tq[q] = in ? T[ck] : R(0);
            Sq[q] = in ? S[ck] : R(0);
            u0q[q] = in ? u[ck] : R(0);
            u1q[q] = in ? u[ck + 1] : R(0);
            v0q[q] = in ? v[ck] : R(0);
            v1q[q] = in ? v[ck + g.pitch] : R(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k4 + q;
            if (k >= nz) break;
            if (k < kb) continue;
            const long ck = k * P + c2;
            const R Tk = Tq[q], Sk = Sq[q];
            const R u0 = u0q[q], u1 = u1q[q], v0 = v0q[q], v1 = v1q[q];
            if (k < nz - 1) {
                R div = dy * p.dz[k] * (u1 - u0) + p.dz[k] * (dxvN * v1 - dxvS * v0);
                wk = wk - div * rac;
                w[ck + P] = wk;
            }
            const R ua = R(0.5) * (u0 + u1), va = R(0.5) * (v0 + v1);
            if (k > kb) {
                R rz = p.rdzf[k];
                R n2 = p.grav * (p.alpha * ((Tk - Tm) + p.dTref[k])
                                 - p.beta_s * ((Sk - Sm) + p.dSref[k])) * rz;
                R s2 = ((ua - ub) * (ua - ub) + (va - vb) * (va - vb)) * rz * rz;
                R kk, nn;
                if (n2 < R(0)) {
                    kk = p.kappa_conv; nn = p.kappa_conv;
                } else {
                    R ri = n2 / (s2 > R(1e-14) ? s2 : R(1e-14));
                    R qr = R(1) + p.ri_a * ri;
                    nn = p.nu0 / (qr * qr) + p.nu_b;
                    kk = nn / qr + p.kappa_b;
                }
                kap[ck] = kk;
                nu[ck] = nn;
            }
            Tm = Tk;
            Sm = Sk;
            ub = ua;
            vb = va;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_diag(KP<R> p, const R* __restrict__ u,
                                              const R* __restrict__ v, const R* __restrict__ T,
                                              const R* __restrict__ S, R* __restrict__ w,
                                              R* __restrict__ pr, R* __restrict__ kap,
                                              R* __restrict__ nu) {
    diag_col<R>(p, (long)blockIdx.x * blockDim.x + threadIdx.x, u, v, T, S, w, pr, kap, nu);
}

// ------------------------------------------------------------------ tile layout

// The tracer and momentum kernels are 2.5-D tiled: a block owns a TX x TY patch of
// columns and marches up through the levels.  Each level's tiles (the patch plus the
// halo its stencils reach, and the patch's own operands) arrive in shared memory by
// tensor copies two levels ahead, in three rotating slots; the block computes every
// face flux / corner vorticity of the level once, one block barrier publishes them and
// frees the slot of the level before, and each thread finishes its own cell.  Vertical
// stencils use a per-thread register window.  The Thomas coefficients of the implicit
// solve go to global scratch (one value per level and column, written and read back by
// the same thread, so they stay in L2).
constexpr int TX = OC_TX, TY = OC_TY, NT = TX * TY;
// rows of the momentum's centred tiles (TY + 1 used), a multiple of 8 so that each slot
// (rows x (TX + 4) FP32 values) is a multiple of 128 bytes
constexpr int PROWS = (TY + 1 + 7) / 8 * 8;
static_assert(TX == 32 && (TY == 8 || TY == 16), "tile shapes the kernels are written for");
static_assert((TY + 8) * (TX + 8) * 4 % 128 == 0 && TY * (TX + 4) * 4 % 128 == 0 &&
              (TY + 1) * TX * 4 % 128 == 0 && TY * TX * 4 % 128 == 0 &&
              PROWS * (TX + 4) * 4 % 128 == 0, "tensor-copy slots on 128-byte boundaries");
// The tracer block has one more warp: its 8 x 33 x-faces and 9 x 32 y-faces (552 WENO
// pairs per level) then take two per thread of 288 instead of up to three of 256; the
// extra warp owns no column and only computes faces.
constexpr int TTY = TY + 1, NTT = TX * TTY;
// resident blocks per SM the register budget is sized for: the FP32 momentum and tracer
// tiles fit 64 and 56 registers (four blocks per SM); the FP64 tiles need far more
template <typename R> struct Occ4 { static constexpr int value = TY == 8 ? 4 : 2; };
template <> struct Occ4<double> { static constexpr int value = 1; };
// the variants with the optional vertical schemes keep more registers: 3 blocks per SM
// of the 32 x 8 tiles.  The momentum tile takes that budget in every form: at 3 blocks
// per SM its FP32 step needs 73 registers and spills none (4.92 -> 4.87 ms at 1/12
// degree, against 4 blocks with 64 registers and a spill); the tracer tile stays at 4
// (6.37 ms against 6.51 at 3 blocks)
template <typename R, bool X> struct OccX { static constexpr int value = X ? (TY == 8 ? 3 : 1) : Occ4<R>::value; };
template <bool X> struct OccX<double, X> { static constexpr int value = 1; };

// padded index of (i, j), clamped into the allocated halo: tiles at the ragged edge of
// the domain stage a few columns beyond it, whose values only feed threads that are
// themselves outside the domain
__device__ __forceinline__ long tix(const GeoD& g, int i, int j) {
    i = i < g.nx + OC_H - 1 ? i : g.nx + OC_H - 1;
    j = j < g.ny + OC_H - 1 ? j : g.ny + OC_H - 1;
    return ix2(g, i, j);
}

// ---- tensor-memory-accelerator copies of tiles, completed on an mbarrier
__device__ int g_tile_err = 0;   // set when a tile's bounded wait gave up

__device__ __forceinline__ unsigned sm_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm_u32(b)));
}
__device__ __forceinline__ void bar_inval(unsigned long long* b) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(sm_u32(b)));
}
__device__ __forceinline__ void bar_expect(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sm_u32(b)),
                 "r"(bytes)
                 : "memory");
}
// one level (z) of a 3-D box at (x, y); x times the element size is a multiple of 16
__device__ __forceinline__ void tma_level(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(sm_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(sm_u32(b))
        : "memory");
}
// waits (at most ~1 s of SM clock) for phase `parity` of the barrier; on giving up it
// flags g_tile_err (the host reports OCEAN_ERR_TIMEOUT) and returns.  Once any wait has
// given up, every later wait that is not satisfied at once returns too, so that a kernel
// whose barriers can no longer complete drains in about one time limit.
__device__ __forceinline__ void bar_wait(unsigned long long* b, unsigned parity) {
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(sm_u32(b)), "r"(parity)
            : "memory");
        if (ok) return;
        if (*reinterpret_cast<volatile int*>(&g_tile_err)) return;
        if (clock64() - t0 > 2000000000LL) {
            atomicExch(&g_tile_err, 1);
            return;
        }
    }
}

// ------------------------------------------------------------------ tracers

// TMA destinations first, each buffer a multiple of 128 bytes: T, S tiles of 14 x 40
// (rows j0-3 .., columns i0-4 ..; rows 14, 15 unused), u faces 8 x 36 (columns i0 ..,
// 33 used), v faces 9 x 32
template <typename R>
struct __align__(128) TracerSmem {
    using R2 = typename Vec2<R>::type;
    R T[3][TY + 8][TX + 8], S[3][TY + 8][TX + 8];     // anomalies of levels k, k+1, k+2
    R us[3][TY][TX + 4], vs[3][TY + 1][TX];           // face velocities of those levels
    R own[3][4][TY][TX];                              // own columns: w(k+1), kap(k+1), G_T(k), G_S(k)
    // x- and y-face transports and (T, S) fluxes of levels k (even) and k+1 (odd)
    R2 fxTS[2][TY][TX + 1], fyTS[2][TY + 1][TX];
    R fxU[2][TY][TX + 1], fyV[2][TY + 1][TX];
    unsigned long long bar[3];                        // buffer b's copies have landed
    short kb[TY + 6][TX + 6];                         // lowest wet level of those columns
    short kbu[TY][TX + 1], kbv[TY + 1][TX];           // lowest wet level of the faces
    // lowest level from which all six cells an x- (y-) face's stencils can touch are wet
    short kfx[TY][TX + 1], kfy[TY + 1][TX];
    int kmin;
};

// STEP = false: G^n of T, S into Tn, Sn.  STEP = true: quasi-AB2 predictor
// T* = T + dt (ca G^n - cb G^{n-1}), G^{n-1} <- G^n, then the backward-Euler diffusion
//   T_k - T*_k = dt/dz_k [kap_{k+1} (T_{k+1} - T_k)/dzf_{k+1} - kap_k (T_k - T_{k-1})/dzf_k]
// with zero flux at the sea floor and the surface, by the Thomas algorithm: forward
// elimination from the bottom while the column is swept upward (c' overwrites kap, d'
// goes to Tn, Sn), back substitution down.  Horizontal fluxes reconstruct the anomalies
// (WENO is translation-equivariant, so adding U Tref(k) gives the flux of T itself);
// vertical ones reconstruct full values, since the reference varies along the column.
// tile (bx, by): columns [bx TX, bx TX + TX) x [by TY, by TY + TY)
// SV: the vertical reconstructions take the stretched-level coefficients of p.vw.
template <typename R, bool STEP, bool SV, typename Off = unsigned>
__device__ __forceinline__ void tracer_tile(const KP<R>& p, const TileMaps& tm, const int bx,
                                            const int by, const TracerArgs<R>& a) {
    using R2 = typename Vec2<R>::type;
    __shared__ TracerSmem<R> sm;
    const GeoD& g = p.g;
    const int nz = g.nz;
    // cell offsets: 32-bit by default (a 3-D array holds fewer than 2^31 cells, checked
    // at creation); the ensemble's tiles keep 64-bit ones, which need fewer registers there
    const Off P = (Off)g.plane;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = bx * TX, j0 = by * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool mine = ty < TY && i < g.nx && j < g.ny;
    const Off c2 = (Off)ix2(g, mine ? i : 0, mine ? j : 0);
    // ---- 2-D masks of the patch, and the lowest wet level of the whole patch
    if (tid == 0) sm.kmin = nz;
    for (int q = tid; q < (TY + 6) * (TX + 6); q += NTT) {
        const int a = q / (TX + 6), b = q % (TX + 6);
        sm.kb[a][b] = g.kb[tix(g, i0 - 3 + b, j0 - 3 + a)];
    }
    for (int q = tid; q < TY * (TX + 1); q += NTT) {
        const int a = q / (TX + 1), b = q % (TX + 1);
        const int fi = i0 + b, fj = j0 + a;
        sm.kbu[a][b] = (fi <= g.nx && fj < g.ny) ? g.kbu[ix2(g, fi, fj)] : (short)nz;
    }
    for (int q = tid; q < (TY + 1) * TX; q += NTT) {
        const int a = q / TX, b = q % TX;
        const int fi = i0 + b, fj = j0 + a;
        sm.kbv[a][b] = (fi < g.nx && fj <= g.ny) ? g.kbv[ix2(g, fi, fj)] : (short)nz;
    }
    __syncthreads();
    const int kb = mine ? (int)sm.kb[ty + 3][tx + 3] : nz;
    if (kb < nz) atomicMin(&sm.kmin, kb);
    for (int q = tid; q < TY * (TX + 1); q += NTT) {
        const int a = q / (TX + 1), b = q % (TX + 1);
        short m = sm.kb[a + 3][b];
#pragma unroll
        for (int n = 1; n < 6; ++n) m = max(m, sm.kb[a + 3][b + n]);
        sm.kfx[a][b] = m;
    }
    for (int q = tid; q < (TY + 1) * TX; q += NTT) {
        const int a = q / TX, b = q % TX;
        short m = sm.kb[a][b + 3];
#pragma unroll
        for (int n = 1; n < 6; ++n) m = max(m, sm.kb[a + n][b + 3]);
        sm.kfy[a][b] = m;
    }
    __syncthreads();
    const int kstart = sm.kmin;
    if (kstart >= nz) return;   // the whole patch is land

    // ---- the staged tile (halo 3) and the face velocities stream in two levels ahead,
    // triple buffered, as tensor copies one thread issues per level (rows and columns
    // beyond the arrays arrive as zeros and feed only threads outside the domain)
    constexpr unsigned STAGE_BYTES =
        (unsigned)sizeof(R) * (2u * (TY + 6) * (TX + 8) + (unsigned)TY * (TX + 4) + (unsigned)(TY + 1) * TX);
    constexpr unsigned OWN_BYTES = (unsigned)sizeof(R) * TY * TX;
    if (tid == 0) {
        bar_init(&sm.bar[0]);
        bar_init(&sm.bar[1]);
        bar_init(&sm.bar[2]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    // with the own columns' operands of the level: a.w and the diffusivity on its top face
    // (level k+1, when there is one), and with STEP G_T and G_S of the previous step
    auto stage = [&](int k, int buf) {
        if (tid == 0) {
            const bool top = k + 1 < nz;
            const unsigned n_own = (top ? 1u : 0u) + (STEP ? (top ? 1u : 0u) + 2u : 0u);
            bar_expect(&sm.bar[buf], STAGE_BYTES + n_own * OWN_BYTES);
            tma_level(&sm.T[buf][0][0], &tm.T, i0, j0 + OC_H - 3, k, &sm.bar[buf]);
            tma_level(&sm.S[buf][0][0], &tm.S, i0, j0 + OC_H - 3, k, &sm.bar[buf]);
            tma_level(&sm.us[buf][0][0], &tm.tu, i0 + OC_H, j0 + OC_H, k, &sm.bar[buf]);
            tma_level(&sm.vs[buf][0][0], &tm.tv, i0 + OC_H, j0 + OC_H, k, &sm.bar[buf]);
            if (top) tma_level(&sm.own[buf][0][0][0], &tm.tw, i0 + OC_H, j0 + OC_H, k + 1, &sm.bar[buf]);
            if (STEP) {
                if (top) tma_level(&sm.own[buf][1][0][0], &tm.tk, i0 + OC_H, j0 + OC_H, k + 1, &sm.bar[buf]);
                tma_level(&sm.own[buf][2][0][0], &tm.tgt, i0 + OC_H, j0 + OC_H, k, &sm.bar[buf]);
                tma_level(&sm.own[buf][3][0][0], &tm.tgs, i0 + OC_H, j0 + OC_H, k, &sm.bar[buf]);
            }
        }
    };
    stage(kstart, 0);
    if (kstart + 1 < nz) stage(kstart + 1, 1);

    const R rac = p.rAc[(mine ? j : 0) + OC_H];
    // register window of full values at levels k-2 .. k+3 (0 outside the column)
    R wT[6], wS[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int kk = kstart - 2 + q;
        const bool ok = mine && kk >= kb && kk < nz;
        wT[q] = ok ? a.T[(Off)kk * P + c2] + p.Tref[kk] : R(0);
        wS[q] = ok ? a.S[(Off)kk * P + c2] + p.Sref[kk] : R(0);
    }
    // anomalies of level kstart+4, the next to enter the window
    R nT, nS;
    {
        const int kk = kstart + 4;
        const bool ok = mine && kk >= kb && kk < nz;
        nT = ok ? a.T[(Off)kk * P + c2] : R(0);
        nS = ok ? a.S[(Off)kk * P + c2] : R(0);
    }
    R fzT = R(0), fzS = R(0), cprev = R(0), dTprev = R(0), dSprev = R(0);
    R kcarry = R(0);   // diffusivity on the top face of the previous level
    int cb = 0;                 // staging slot of level k: (k - kstart) mod 3
    unsigned phase = 0;         // bit s: parity of slot s's next completion

    // One block barrier per level: the faces of level k go to face buffer k & 1, so a
    // warp that has finished level k-1 computes level k's faces while others still read
    // level k-1's; the barrier after the faces publishes them and frees the staging
    // buffer of level k-1 (read by every thread before it), which takes level k+2.
    // the y-faces' row metric: row ty (row TY for the extra warp) on every level
    const R dxv = p.dxv[j0 + (ty < TY ? ty : TY) + OC_H];
    for (int k = kstart; k < nz; ++k) {
        const Off Pk = (Off)k * P;
        const int fb = (k - kstart) & 1;
        bar_wait(&sm.bar[cb], (phase >> cb) & 1u);
        phase ^= 1u << cb;
        const R dzk = __ldg(p.lvt + (size_t)k * OC_LVROW);   // dz of the level (row k, first value)
        // ---- x- and y-face fluxes, each face once, by fixed roles: thread (tx, ty < TY)
        // the west and south faces of its own column; the extra warp the north faces of the last row and (lanes 0..TY-1) the east faces
        // of the last column.  Two WENO pairs per thread; the stencil offsets are known at
        // compile time.
        auto xface = [&](const int a, const int b) {
            R fU = R(0), fT = R(0), fS = R(0);
            const bool full = k >= sm.kfx[a][b];   // every stencil point wet
            if (full || k >= sm.kbu[a][b]) {
                const R ut = sm.us[cb][a][b];
                const bool pos = ut >= R(0);
                // upwind to downwind: columns b .. b+4 (ut >= 0) or b+5 .. b+1
                const R* tT = &sm.T[cb][a + 3][pos ? b + 1 : b + 6];
                const R* tS = &sm.S[cb][a + 3][pos ? b + 1 : b + 6];
                const int st = pos ? 1 : -1;
                R qT[5], qS[5];
                unsigned in = full ? 31u : 0u;
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    qT[n] = tT[n * st];
                    qS[n] = tS[n * st];
                    if (!full) {
                        const int col = pos ? b + n : b + 5 - n;
                        in |= (k >= sm.kb[a + 3][col] ? 1u : 0u) << n;
                    }
                }
                R rT, rS;
                WenoPair<R>::run(qT, qS, in, in, p.eps, p.linear, rT, rS);
                fU = ut * p.dy * dzk;
                fT = fU * rT;
                fS = fU * rS;
            }
            sm.fxU[fb][a][b] = fU;
            sm.fxTS[fb][a][b] = make_vec2(fT, fS);
        };
        auto yface = [&](const int a, const int b) {
            R fV = R(0), fT = R(0), fS = R(0);
            const bool full = k >= sm.kfy[a][b];
            if (full || k >= sm.kbv[a][b]) {
                const R vt = sm.vs[cb][a][b];
                const bool pos = vt >= R(0);
                // rows a .. a+4 (vt >= 0) or a+5 .. a+1
                const R* tT = &sm.T[cb][pos ? a : a + 5][b + 4];
                const R* tS = &sm.S[cb][pos ? a : a + 5][b + 4];
                const int st = pos ? (TX + 8) : -(TX + 8);
                R qT[5], qS[5];
                unsigned in = full ? 31u : 0u;
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    qT[n] = tT[n * st];
                    qS[n] = tS[n * st];
                    if (!full) {
                        const int row = pos ? a + n : a + 5 - n;
                        in |= (k >= sm.kb[row][b + 3] ? 1u : 0u) << n;
                    }
                }
                R rT, rS;
                WenoPair<R>::run(qT, qS, in, in, p.eps, p.linear, rT, rS);
                fV = vt * dxv * dzk;
                fT = fV * rT;
                fS = fV * rS;
            }
            sm.fyV[fb][a][b] = fV;
            sm.fyTS[fb][a][b] = make_vec2(fT, fS);
        };
        if (ty < TY) {
            xface(ty, tx);
            yface(ty, tx);
        } else {
            yface(TY, tx);
            if (tx < TY) xface(tx, TX);
        }
        // this thread's reads of level k-1's staging buffer (faces and own cell, before
        // this point) are ordered before the tensor copy that overwrites it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        const int c2s = cb == 0 ? 2 : cb - 1;   // slot of level k+2: (k - kstart + 2) mod 3
        if (k + 2 < nz) stage(k + 2, c2s);
        // own-cell operands of level k, from its staging slot (rewritten only by the copy of
        // level k+3, issued after the next level's barrier); the diffusivity on the bottom
        // face is the previous level's top one
        const bool live = mine && k >= kb;
        const Off ck = Pk + c2;
        R wt = R(0), k0 = kcarry, k1 = R(0), gT0 = R(0), gS0 = R(0), T0 = R(0), S0 = R(0);
        if (live) {
            if (k + 1 < nz) {
                wt = sm.own[cb][0][ty][tx];
                if (STEP) k1 = sm.own[cb][1][ty][tx];
            }
            if (STEP) {
                gT0 = sm.own[cb][2][ty][tx];
                gS0 = sm.own[cb][3][ty][tx];
                T0 = sm.T[cb][ty + 3][tx + 4];
                S0 = sm.S[cb][ty + 3][tx + 4];
            }
        }
        kcarry = k1;
        // ---- own cell
        if (live) {
            // level constants (row k of the level table, read where used): 1/dz, the
            // implicit solve's off-diagonal factors dt/(dz dzf) below and above, Tref, Sref
            // and the diffusion of the reference profiles
            const R* L = p.lvt + (size_t)k * OC_LVROW;
            R ftT = R(0), ftS = R(0);
            if (k + 1 < nz) {   // flux through the top face (bottom face of cell k+1)
                const bool pos = wt >= R(0);
                // all five levels of the stencil in the column: k-2..k+2 upward, k-1..k+3
                // downward
                const bool full = pos ? (k - 2 >= kb && k + 2 < nz) : (k - 1 >= kb && k + 3 < nz);
                R qT[5], qS[5];
                unsigned in = full ? 31u : 0u;
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    // window index n (level k-2+n) upward, 5-n (level k+3-n) downward; both
                    // compile-time so the window stays in registers
                    qT[n] = pos ? wT[n] : wT[5 - n];
                    qS[n] = pos ? wS[n] : wS[5 - n];
                    const int kk = pos ? k - 2 + n : k + 3 - n;
                    if (!full) in |= (kk >= kb && kk < nz ? 1u : 0u) << n;
                }
                R rT, rS;
                if (SV) {
                    const R* row = p.vw + ((k + 1) * 2 + (pos ? 0 : 1)) * OC_VWROW;
                    WenoPairRow<R>::run(qT, qS, in, in, row, row, p.eps, p.linear, rT, rS);
                } else {
                    WenoPair<R>::run(qT, qS, in, in, p.eps, p.linear, rT, rS);
                }
                ftT = wt * rT;
                ftS = wt * rS;
            }
            const R rdz = __ldg(L + 1);
            const R eU = sm.fxU[fb][ty][tx + 1], nV = sm.fyV[fb][ty + 1][tx];
            const R wU = sm.fxU[fb][ty][tx], sV = sm.fyV[fb][ty][tx];
            const R2 eTS = sm.fxTS[fb][ty][tx + 1], nTS = sm.fyTS[fb][ty + 1][tx];
            const R2 wTS = sm.fxTS[fb][ty][tx], sTS = sm.fyTS[fb][ty][tx];
            const R divU = eU - wU + nV - sV;
            const R hT = eTS.x - wTS.x + nTS.x - sTS.x;
            const R hS = eTS.y - wTS.y + nTS.y - sTS.y;
            R GT = -((__ldg(L + 4) * divU + hT) * rac + (ftT - fzT)) * rdz;
            R GS = -((__ldg(L + 5) * divU + hS) * rac + (ftS - fzS)) * rdz;
            if (a.dGT) {   // learned-closure corrections, part of G^n
                GT += a.dGT[ck];
                GS += a.dGS[ck];
            }
            fzT = ftT;
            fzS = ftS;
            if (!STEP) {
                a.Tn[ck] = GT;
                a.Sn[ck] = GS;
            } else {
                const R gT = p.ca * GT - p.cb * gT0;
                const R gS = p.ca * GS - p.cb * gS0;
                a.GTp[ck] = GT;
                a.GSp[ck] = GS;
                // lo, hi: dt a.kap / (dz dzf) on the bottom and top faces (zero at the ends)
                const R lo = k > kb ? k0 * __ldg(L + 2) : R(0);
                const R hi = k1 * __ldg(L + 3);   // a.kap on the surface face is zero
                // the diffusion of the reference profile moves to the right-hand side:
                // (I - dt D) a.T'^{n+1} = a.T'* + dt D Tref
                const R Ts = T0 + p.dt * gT + k1 * __ldg(L + 6) - (k > kb ? k0 * __ldg(L + 7) : R(0));
                const R Ss = S0 + p.dt * gS + k1 * __ldg(L + 8) - (k > kb ? k0 * __ldg(L + 9) : R(0));
                const R inv = rcp_pivot((R(1) + lo + hi) + lo * cprev);   // b_k - a_k c'_{k-1}
                cprev = -hi * inv;
                dTprev = (Ts + lo * dTprev) * inv;
                dSprev = (Ss + lo * dSprev) * inv;
                a.kap[ck] = cprev;
                a.Tn[ck] = dTprev;
                a.Sn[ck] = dSprev;
            }
        }
        cb = cb == 2 ? 0 : cb + 1;
        // ---- slide the vertical window up one level
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            wT[q] = wT[q + 1];
            wS[q] = wS[q + 1];
        }
        {
            // level k+4 enters from the anomalies loaded one level earlier (their memory
            // latency hidden behind that level's work); level k+5's are loaded now
            const int kk = k + 4;
            const bool ok = mine && kk >= kb && kk < nz;
            wT[5] = ok ? nT + p.Tref[kk] : R(0);
            wS[5] = ok ? nS + p.Sref[kk] : R(0);
            const bool ok5 = mine && kk + 1 >= kb && kk + 1 < nz;
            nT = ok5 ? a.T[(Off)(kk + 1) * P + c2] : R(0);
            nS = ok5 ? a.S[(Off)(kk + 1) * P + c2] : R(0);
        }
    }
    __syncthreads();   // every copy waited for: the barriers can be retired
    if (tid == 0) {
        bar_inval(&sm.bar[0]);
        bar_inval(&sm.bar[1]);
        bar_inval(&sm.bar[2]);
    }
    if (!STEP || !mine || kb >= nz) return;
    // back substitution down the column, the coefficients of four levels loaded at once
    // (the recurrence itself is serial)
    R xT = dTprev, xS = dSprev;   // level nz-1: x = d'
    for (int k = nz - 2; k >= kb; k -= 4) {
        R cc[4], tq[4], sq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Off ck = (Off)(k - q) * P + c2;
            const bool in = k - q >= kb;
            cc[q] = in ? a.kap[ck] : R(0);
            tq[q] = in ? a.Tn[ck] : R(0);
            sq[q] = in ? a.Sn[ck] : R(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (k - q < kb) break;
            const Off ck = (Off)(k - q) * P + c2;
            xT = tq[q] - cc[q] * xT;
            xS = sq[q] - cc[q] * xS;
            a.Tn[ck] = xT;
            a.Sn[ck] = xS;
        }
    }
}

template <typename R, bool STEP, bool SV>
__global__ void __launch_bounds__(NTT, (OccX<R, SV>::value)) k_tracer(
    KP<R> p, const __grid_constant__ TileMaps tm, const __grid_constant__ TracerArgs<R> a) {
    tracer_tile<R, STEP, SV>(p, tm, blockIdx.x, blockIdx.y, a);
}

// ------------------------------------------------------------------ momentum

// TMA destinations first, each buffer a multiple of 128 bytes; every box starts at the
// column i0-4 (16-byte aligned), so the logical column c of each array sits at c + 2 (u),
// c + 1 (v), c + 3 (p, w, nu).  Slot s holds one level's tiles; three slots rotate.
template <typename R>
struct __align__(128) MomentumSmem {
    R u[3][TY + 8][TX + 8];   // u at i in [i0-2, i0+TX+3), j in [j0-3, j0+TY+3)
    R v[3][TY + 8][TX + 8];   // v at i in [i0-3, i0+TX+3), j in [j0-2, j0+TY+3)
    R p[3][PROWS][TX + 4];   // pressure anomaly at centres i in [i0-1, i0+TX), j in [j0-1, j0+TY)
    R w[3][PROWS][TX + 4];   // w on the level's bottom faces, same centres
    R nu[3][PROWS][TX + 4];  // nu on those faces
    R gu[3][TY][TX], gv[3][TY][TX];   // own columns' G_u, G_v of the previous step
    unsigned long long bar[3];        // slot s's copies have landed
    // corner vorticity, i in [i0-2, i0+TX+3), j in [j0-2, j0+TY+3), and the kinetic energy
    // at the centres, of levels k (even) and k+1 (odd)
    R z[2][TY + 5][TX + 5];
    R K[2][TY + 1][TX + 1];
    short kbz[TY + 5][TX + 5], kbzin[TY + 5][TX + 5];
    R zdxS[TY + 5], zdxN[TY + 5], zrA[TY + 5];   // per corner row: dxc south, north; 1/A_z
    int kmin;
};

// STEP = false: G^n of u, v into un, vn.  STEP = true: quasi-AB2 predictor, G^{n-1} <-
// G^n, the column sums U^n = sum dz u^n and G_U = sum dz G^ of the barotropic mode, the
// backward-Euler vertical viscosity (Thomas: c' in cu/cv scratch, d' in un/vn) and the
// sum of the solved column Su = sum dz u**.  VA: the vertical advection in the WENO flux
// form (own-column windows of u and v over levels k-2 .. k+3 in registers, the bottom
// face's flux carried up from the level below), else centred.
template <typename R, bool STEP, bool VA, typename Off = unsigned>
__device__ __forceinline__ void momentum_tile(const KP<R>& p, const TileMaps& tm, const int bx,
                                              const int by, const MomentumArgs<R>& a) {
    __shared__ MomentumSmem<R> sm;
    const GeoD& g = p.g;
    const int nz = g.nz;
    // cell offsets: 32-bit by default (a 3-D array holds fewer than 2^31 cells, checked
    // at creation); the ensemble's tiles keep 64-bit ones, which need fewer registers there
    const Off P = (Off)g.plane;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = bx * TX, j0 = by * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool mine = i < g.nx && j < g.ny;
    const Off c2 = (Off)ix2(g, mine ? i : 0, mine ? j : 0);
    if (tid == 0) sm.kmin = nz;
    for (int q = tid; q < (TY + 5) * (TX + 5); q += NT) {
        const int a = q / (TX + 5), b = q % (TX + 5);
        const long c = tix(g, i0 - 2 + b, j0 - 2 + a);
        sm.kbz[a][b] = g.kbz[c];
        sm.kbzin[a][b] = g.kbzin[c];
    }
    if (tid < TY + 5) {
        const int jc = j0 - 2 + tid;
        const int jrc = (jc < g.ny + OC_H - 1 ? jc : g.ny + OC_H - 1) + OC_H;
        sm.zdxS[tid] = p.dxc[jrc - 1];
        sm.zdxN[tid] = p.dxc[jrc];
        sm.zrA[tid] = p.rAz[jrc];
    }
    const int ku = mine ? (int)g.kbu[c2] : nz, kv = mine ? (int)g.kbv[c2] : nz;
    __syncthreads();
    const int k0 = ku < kv ? ku : kv;
    if (k0 < nz) atomicMin(&sm.kmin, k0);
    __syncthreads();
    const int kstart = sm.kmin;
    if (kstart >= nz) return;

    // ---- staging by tensor copies one thread issues: level k's a.u, a.v, p, a.w, a.nu tiles (and
    // with STEP its own columns' G^{n-1}) into slot (k - kstart) % 3, two levels ahead.
    // Level k's own cells read its slot and level k+1's (a.u, a.v above, a.w and a.nu on the top
    // face).
    constexpr int TC = (TY + 1) * (TX + 1);   // centres of the pressure / a.w / a.nu tiles
    constexpr unsigned TILES = (unsigned)sizeof(R) * ((TX + 8) * (TY + 6) + (TX + 8) * (TY + 5) +
                                                      3u * (TX + 4) * (TY + 1));
    constexpr unsigned OWN = (unsigned)sizeof(R) * TY * TX;
    const int yu = j0 + OC_H - 3, yv = j0 + OC_H - 2, yc = j0 + OC_H - 1;
    auto stage = [&](int k, int sl) {
        unsigned long long* bar = &sm.bar[sl];
        bar_expect(bar, TILES + (STEP ? 2u * OWN : 0u));
        tma_level(&sm.u[sl][0][0], &tm.mu, i0, yu, k, bar);
        tma_level(&sm.v[sl][0][0], &tm.mv, i0, yv, k, bar);
        tma_level(&sm.p[sl][0][0], &tm.mp, i0, yc, k, bar);
        tma_level(&sm.w[sl][0][0], &tm.mw, i0, yc, k, bar);
        tma_level(&sm.nu[sl][0][0], &tm.mnu, i0, yc, k, bar);
        if (STEP) {
            tma_level(&sm.gu[sl][0][0], &tm.mgu, i0 + OC_H, j0 + OC_H, k, bar);
            tma_level(&sm.gv[sl][0][0], &tm.mgv, i0 + OC_H, j0 + OC_H, k, bar);
        }
    };
    if (tid == 0) {
        bar_init(&sm.bar[0]);
        bar_init(&sm.bar[1]);
        bar_init(&sm.bar[2]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        stage(kstart, 0);
        if (kstart + 1 < nz) stage(kstart + 1, 1);
    }
    __syncthreads();   // the barriers are initialised before anyone waits on them

    const int jr = (mine ? j : 0) + OC_H;
    const R rdxc = p.rdxc[jr], fu = p.fu[jr], fv = p.fv[jr];
    // the corners and kinetic-energy centres this thread computes on every level: fixed
    // for the whole march (two slots each; the second only for the first threads), so
    // their indices, shared-memory offsets and corner masks are formed once
    constexpr int NCR = (TY + 5) * (TX + 5);
    static_assert(NCR <= 2 * NT && TC <= 2 * NT, "two corner and two centre slots per thread");
    // the lowest level from which all six corners of this thread's a.u-face (a.v-face)
    // vorticity stencils touch the fluid
    int kzu = 0, kzv = 0;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
        kzu = max(kzu, (int)sm.kbzin[ty + n][tx + 2]);
        kzv = max(kzv, (int)sm.kbzin[ty + 2][tx + n]);
    }
    // corner slot (-1: none): its offset in a level's u / v tile (row a, column b) in bits
    // 0..9, in the vorticity buffer in bits 10..18, the row a in bits 19..22 and its lowest
    // active level from bit 23; centre slot (-1: none): the offset of u(row a + 2, column
    // b + 3) in a u / v tile in bits 0..9, of the centre in the kinetic-energy buffer from
    // bit 10
    static_assert((TY + 4) * (TX + 8) + TX + 4 < 1024 && (TY + 5) * (TX + 5) < 512 && TY + 5 <= 16 &&
                  OC_NZMAX < 256 && (TY + 1) * (TX + 1) < (1 << 20), "slot fields");
    auto zslot = [&](int q) {
        if (q >= NCR) return -1;
        const int a = q / (TX + 5), b = q % (TX + 5);
        return (a * (TX + 8) + b) | ((a * (TX + 5) + b) << 10) | (a << 19) | ((int)sm.kbz[a][b] << 23);
    };
    auto kslot = [&](int q) {
        if (q >= TC) return -1;
        const int a = q / (TX + 1), b = q % (TX + 1);
        return ((a + 2) * (TX + 8) + b + 3) | ((a * (TX + 1) + b) << 10);
    };
    const int zs0 = zslot(tid), zs1 = zslot(tid + NT), ko0 = kslot(tid), ko1 = kslot(tid + NT);
    R sUn = 0, sGU = 0, sVn = 0, sGV = 0;
    R cuk = 0, duk = 0, cvk = 0, dvk = 0;
    // carried up one level: the vertical advection through the top face (the next
    // level's bottom-face term) and the sum of the two a.nu on the top face
    R upu = R(0), upv = R(0), nsu = R(0), nsv = R(0);
    // WENO vertical advection: own a.u- and a.v-face values at levels k-2 .. k+3 (0 outside
    // the face's wet levels), and the flux and a.w of the bottom face
    R wu[6], wv[6];
    R fbu = R(0), fbv = R(0), wbu = R(0), wbv = R(0);
    if (VA) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int kk = kstart - 2 + q;
            wu[q] = mine && kk >= ku && kk < nz ? a.u[(Off)kk * P + c2] : R(0);
            wv[q] = mine && kk >= kv && kk < nz ? a.v[(Off)kk * P + c2] : R(0);
        }
    }
    int r3 = 0, q3 = 0;   // (k - kstart) mod 3 and div 3
    // One block barrier per level: corners and kinetic energy of level k go to buffer
    // k & 1, so a warp that has finished level k-1 computes them while others still read
    // level k-1's; the barrier after them publishes them and frees the slot of level k-1
    // (read by every thread before it), which takes level k+2.
    for (int k = kstart; k < nz; ++k) {
        const Off Pk = (Off)k * P;
        // slots of levels k, k+1, k+2 and the parities of their completions, from the
        // running quotient and remainder of (k - kstart) / 3
        const int sc = r3, sn = r3 == 2 ? 0 : r3 + 1, s2 = r3 == 0 ? 2 : r3 - 1, fb = (k - kstart) & 1;
        const unsigned pc = (unsigned)q3 & 1u, pn = (unsigned)(r3 == 2 ? q3 + 1 : q3) & 1u;
        bar_wait(&sm.bar[sc], pc);
        // ---- corner vorticity (zero unless all four cells are wet) and kinetic energy
        const R* const ul = &sm.u[sc][0][0];
        const R* const vl = &sm.v[sc][0][0];
        auto corner = [&](const int zsr) {
            const int a = (zsr >> 19) & 15;
            const R* us = ul + (zsr & 1023);
            const R* vs = vl + (zsr & 1023);
            R zz = R(0);
            if (k >= (zsr >> 23)) {
                // a.u(i, jc) = a.u[a + 1][b], a.u(i, jc-1) = a.u[a][b]; a.v(i, jc) = a.v[a][b + 1],
                // a.v(i-1, jc) = a.v[a][b]  (tile columns offset by 2 for a.u, 1 for a.v)
                const R circ = p.dy * (vs[2] - vs[1])
                             - (sm.zdxN[a] * us[(TX + 8) + 2] - sm.zdxS[a] * us[2]);
                zz = circ * sm.zrA[a];
            }
            (&sm.z[fb][0][0])[(zsr >> 10) & 511] = zz;
        };
        corner(zs0);
        if (zs1 >= 0) corner(zs1);
        auto centre = [&](const int kor) {
            // centre (i0-1+b, j0-1+a): a.u at cols b+1, b+2 of row a+2; a.v at col b+2, rows
            // a+1, a+2 (tile columns offset by 2 for a.u, 1 for a.v: the same tile offset)
            const int o = kor & 1023;
            const R ua = ul[o], ub = ul[o + 1];
            const R va = vl[o - (TX + 8)], vb = vl[o];
            (&sm.K[fb][0][0])[kor >> 10] = R(0.25) * (ua * ua + ub * ub) + R(0.25) * (va * va + vb * vb);
        };
        centre(ko0);
        if (ko1 >= 0) centre(ko1);
        // this thread's reads of level k-1's slot are ordered before the tensor copy that
        // overwrites it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0 && k + 2 < nz) stage(k + 2, s2);
        if (k + 1 < nz) bar_wait(&sm.bar[sn], pn);
        if (mine) {
            // level constants (row k of the level table, read where used): dz, 1/dz and the
            // implicit solve's factors dt/(dz dzf) below and above
            const R* L = p.lvt + (size_t)k * OC_LVROW;
            const R rdz = __ldg(L + 1);
            const bool du_ = k >= ku, dv_ = k >= kv;
            const R uhi = k + 1 < nz ? sm.u[sn][ty + 3][(tx + 2) + 2] : R(0);
            const R vhi = k + 1 < nz ? sm.v[sn][ty + 2][(tx + 3) + 1] : R(0);
            const R gu0 = STEP && du_ ? sm.gu[sc][ty][tx] : R(0);
            const R gv0 = STEP && dv_ ? sm.gv[sc][ty][tx] : R(0);
            // ---- the two vorticity reconstructions of this thread
            const R u0 = sm.u[sc][ty + 3][(tx + 2) + 2];
            const R v0 = sm.v[sc][ty + 2][(tx + 3) + 1];
            const R vh = R(0.25) * (sm.v[sc][ty + 2][(tx + 2) + 1] + sm.v[sc][ty + 2][(tx + 3) + 1]
                                  + sm.v[sc][ty + 3][(tx + 2) + 1] + sm.v[sc][ty + 3][(tx + 3) + 1]);
            const R uh = R(0.25) * (sm.u[sc][ty + 2][(tx + 2) + 2] + sm.u[sc][ty + 2][(tx + 3) + 2]
                                  + sm.u[sc][ty + 3][(tx + 2) + 2] + sm.u[sc][ty + 3][(tx + 3) + 2]);
            R qa[5], qb[5];
            // upwind to downwind: corner rows j-2 .. j+2 (vh >= 0) or j+3 .. j-1 at the
            // a.u-face's column; corner columns i-2 .. i+2 (uh >= 0) or i+3 .. i-1 on the
            // a.v-face's row.  A stencil whose six corners all touch the fluid needs no mask.
            const bool pa = vh >= R(0), pb = uh >= R(0);
            const R* za = &sm.z[fb][pa ? ty : ty + 5][tx + 2];
            const R* zb = &sm.z[fb][ty + 2][pb ? tx : tx + 5];
            const int sa = pa ? (TX + 5) : -(TX + 5), sb = pb ? 1 : -1;
            const bool fa = k >= kzu, fbb = k >= kzv;
            unsigned ina = fa ? 31u : 0u, inb = fbb ? 31u : 0u;
#pragma unroll
            for (int n = 0; n < 5; ++n) {
                qa[n] = za[n * sa];
                qb[n] = zb[n * sb];
            }
            if (!fa) {
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    const int a = pa ? ty + n : ty + 5 - n;
                    ina |= (k >= sm.kbzin[a][tx + 2] ? 1u : 0u) << n;
                }
            }
            if (!fbb) {
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    const int b = pb ? tx + n : tx + 5 - n;
                    inb |= (k >= sm.kbzin[ty + 2][b] ? 1u : 0u) << n;
                }
            }
            R ztu, ztv;
            WenoPair<R>::run(qa, qb, ina, inb, p.eps, p.linear, ztu, ztv);
            // WENO flux form of the vertical advection:
            // [w_top a.u~_top - w_bot a.u~_bot - u_k (w_top - w_bot)] / dz_k, a.u~ upwind by a.w
            R vau = R(0), vav = R(0);
            if (VA) {
                R wtu = R(0), wtv = R(0), ftu = R(0), ftv = R(0);
                if (k + 1 < nz) {
                    wtu = R(0.5) * (sm.w[sn][ty + 1][(tx) + 3] + sm.w[sn][ty + 1][(tx + 1) + 3]);
                    wtv = R(0.5) * (sm.w[sn][ty][(tx + 1) + 3] + sm.w[sn][ty + 1][(tx + 1) + 3]);
                    const bool pu = wtu >= R(0), pv = wtv >= R(0);
                    R ra[5], rb[5];
                    unsigned ia = 0, ib = 0;
#pragma unroll
                    for (int n = 0; n < 5; ++n) {
                        // window index n (level k-2+n) upward, 5-n (level k+3-n) downward
                        ra[n] = pu ? wu[n] : wu[5 - n];
                        rb[n] = pv ? wv[n] : wv[5 - n];
                        const int la = pu ? k - 2 + n : k + 3 - n, lb = pv ? k - 2 + n : k + 3 - n;
                        ia |= (la >= ku && la < nz ? 1u : 0u) << n;
                        ib |= (lb >= kv && lb < nz ? 1u : 0u) << n;
                    }
                    R xu, xv;
                    if (p.vweno)
                        WenoPairRow<R>::run(ra, rb, ia, ib, p.vw + ((k + 1) * 2 + (pu ? 0 : 1)) * OC_VWROW,
                                            p.vw + ((k + 1) * 2 + (pv ? 0 : 1)) * OC_VWROW, p.eps,
                                            p.linear, xu, xv);
                    else
                        WenoPair<R>::run(ra, rb, ia, ib, p.eps, p.linear, xu, xv);
                    ftu = wtu * xu;
                    ftv = wtv * xv;
                }
                const bool bu = k > ku, bv = k > kv;   // faces below the lowest wet level carry nothing
                vau = (ftu - (bu ? fbu : R(0)) - u0 * (wtu - (bu ? wbu : R(0)))) * rdz;
                vav = (ftv - (bv ? fbv : R(0)) - v0 * (wtv - (bv ? wbv : R(0)))) * rdz;
                fbu = ftu; wbu = wtu; fbv = ftv; wbv = wtv;
            }
            if (du_) {   // ---------------- a.u at the west face of column (i, j)
                const R dK = (sm.K[fb][ty + 1][tx + 1] - sm.K[fb][ty + 1][tx]) * rdxc;
                const R dP = (sm.p[sc][ty + 1][(tx + 1) + 3] - sm.p[sc][ty + 1][(tx) + 3]) * rdxc;
                R vadv = vau;
                if (!VA) {
                    R up = R(0);
                    if (k + 1 < nz)
                        up = R(0.5) * (sm.w[sn][ty + 1][(tx) + 3] + sm.w[sn][ty + 1][(tx + 1) + 3]) * (uhi - u0) * p.rdzf[k + 1];
                    const R dn = k - 1 >= ku ? upu : R(0);   // the level below's top-face term
                    upu = up;
                    vadv = R(0.5) * (up + dn);
                }
                const R wind = k == nz - 1 ? a.taux_s[c2] : R(0);
                const R G = (ztu + fu) * vh - dK - vadv - dP + wind;
                const Off ck = Pk + c2;
                if (!STEP) {
                    a.un[ck] = G;
                } else {
                    const R gh = p.ca * G - p.cb * gu0;
                    a.Gup[ck] = G;
                    sUn += __ldg(L) * u0;
                    sGU += __ldg(L) * gh;
                    const R us = u0 + p.dt * gh;
                    const R nt = k < nz - 1 ? sm.nu[sn][ty + 1][(tx) + 3] + sm.nu[sn][ty + 1][(tx + 1) + 3] : R(0);
                    const R lo = k > ku ? R(0.5) * nsu * __ldg(L + 2) : R(0);
                    const R hi = R(0.5) * nt * __ldg(L + 3);   // zero at the surface
                    nsu = nt;
                    const R inv = rcp_pivot((R(1) + lo + hi) + lo * cuk);
                    cuk = -hi * inv;
                    duk = (us + lo * duk) * inv;
                    a.cu[ck] = cuk;
                    a.un[ck] = duk;
                }
            }
            if (dv_) {   // ---------------- a.v at the south face of column (i, j)
                const R dK = (sm.K[fb][ty + 1][tx + 1] - sm.K[fb][ty][tx + 1]) * p.rdy;
                const R dP = (sm.p[sc][ty + 1][(tx + 1) + 3] - sm.p[sc][ty][(tx + 1) + 3]) * p.rdy;
                R vadv = vav;
                if (!VA) {
                    R up = R(0);
                    if (k + 1 < nz)
                        up = R(0.5) * (sm.w[sn][ty][(tx + 1) + 3] + sm.w[sn][ty + 1][(tx + 1) + 3]) * (vhi - v0) * p.rdzf[k + 1];
                    const R dn = k - 1 >= kv ? upv : R(0);
                    upv = up;
                    vadv = R(0.5) * (up + dn);
                }
                const R wind = k == nz - 1 ? a.tauy_s[c2] : R(0);
                const R G = -(ztv + fv) * uh - dK - vadv - dP + wind;
                const Off ck = Pk + c2;
                if (!STEP) {
                    a.vn[ck] = G;
                } else {
                    const R gh = p.ca * G - p.cb * gv0;
                    a.Gvp[ck] = G;
                    sVn += __ldg(L) * v0;
                    sGV += __ldg(L) * gh;
                    const R vs = v0 + p.dt * gh;
                    const R nt = k < nz - 1 ? sm.nu[sn][ty][(tx + 1) + 3] + sm.nu[sn][ty + 1][(tx + 1) + 3] : R(0);
                    const R lo = k > kv ? R(0.5) * nsv * __ldg(L + 2) : R(0);
                    const R hi = R(0.5) * nt * __ldg(L + 3);   // zero at the surface
                    nsv = nt;
                    const R inv = rcp_pivot((R(1) + lo + hi) + lo * cvk);
                    cvk = -hi * inv;
                    dvk = (vs + lo * dvk) * inv;
                    a.cv[ck] = cvk;
                    a.vn[ck] = dvk;
                }
            }
        }
        if (VA) {   // slide the windows up one level
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                wu[q] = wu[q + 1];
                wv[q] = wv[q + 1];
            }
            const int kk = k + 4;
            wu[5] = mine && kk >= ku && kk < nz ? a.u[(Off)kk * P + c2] : R(0);
            wv[5] = mine && kk >= kv && kk < nz ? a.v[(Off)kk * P + c2] : R(0);
        }
        if (++r3 == 3) {
            r3 = 0;
            ++q3;
        }
    }
    __syncthreads();   // every copy waited for: the barriers can be retired
    if (tid == 0) {
        bar_inval(&sm.bar[0]);
        bar_inval(&sm.bar[1]);
        bar_inval(&sm.bar[2]);
    }
    if (!STEP || !mine) return;
    // back substitutions of a.u and a.v down the column together, both coefficients of four
    // levels loaded at once (each recurrence itself is serial)
    R xu = duk, xv = dvk;   // level nz-1: x = d'
    R su = p.dz[nz - 1] * xu, sv = p.dz[nz - 1] * xv;
    const int kf = ku < kv ? ku : kv;
    for (int k = nz - 2; k >= kf; k -= 4) {
        R cuq[4], duq[4], cvq[4], dvq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Off ck = (Off)(k - q) * P + c2;
            const bool inu = k - q >= ku, inv = k - q >= kv;
            cuq[q] = inu ? a.cu[ck] : R(0);
            duq[q] = inu ? a.un[ck] : R(0);
            cvq[q] = inv ? a.cv[ck] : R(0);
            dvq[q] = inv ? a.vn[ck] : R(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Off ck = (Off)(k - q) * P + c2;
            if (k - q >= ku) {
                xu = duq[q] - cuq[q] * xu;
                a.un[ck] = xu;
                su += p.dz[k - q] * xu;
            }
            if (k - q >= kv) {
                xv = dvq[q] - cvq[q] * xv;
                a.vn[ck] = xv;
                sv += p.dz[k - q] * xv;
            }
        }
    }
    if (ku < nz) {
        a.Un[c2] = sUn;
        a.GU[c2] = sGU;
        a.Su[c2] = su;
    }
    if (kv < nz) {
        a.Vn[c2] = sVn;
        a.GV[c2] = sGV;
        a.Sv[c2] = sv;
    }
}

template <typename R, bool STEP, bool VA>
__global__ void __launch_bounds__(NT, (OccX<R, true>::value)) k_momentum(
    KP<R> p, const __grid_constant__ TileMaps tm, const __grid_constant__ MomentumArgs<R> a) {
    momentum_tile<R, STEP, VA>(p, tm, blockIdx.x, blockIdx.y, a);
}

// ------------------------------------------------------------------ barotropic mode

// start of the sub-cycle: U^0 = U^n, deta^0 = 0, accumulators cleared, the gradient of
// the FP64 free surface eta^n formed once (in R)
// The sub-cycle's sums over all passes, per column: FP64 words in the FP64 form; in the
// mixed form FP32 words in the first half of the same storage (half the accumulators'
// DRAM traffic per pass; the sums are of deviations from the step's start, O(1e-3) of
// the state, so FP32's 24 bits over ten passes stay far below the mixed form's error).
// A pass adds its partial sums by in-memory reductions: one thread owns each cell, so
// the reduction is the plain add, issued without waiting for the old value.
__device__ __forceinline__ void acc_add(double* a, long c, double p) { atomicAdd(a + c, p); }
__device__ __forceinline__ void acc_add(double* a, long c, float p) {
    atomicAdd(reinterpret_cast<float*>(a) + c, p);
}
template <typename R> __device__ __forceinline__ void acc_zero(double* a, long c) {
    if (sizeof(R) == sizeof(float)) reinterpret_cast<float*>(a)[c] = 0.f;
    else a[c] = 0.0;
}
// an accumulator times s, in the path's precision (FP32 in the mixed form: no FP64 unit)
template <typename R> __device__ __forceinline__ R acc_scaled(const double* a, long c, double s) {
    if (sizeof(R) == sizeof(float)) return (R)(reinterpret_cast<const float*>(a)[c] * (float)s);
    return (R)(a[c] * s);
}

template <typename R>
__device__ __forceinline__ void baro_begin_col(const KP<R>& p, const long c,
                                               const R* __restrict__ Un, const R* __restrict__ Vn,
                                               const double* __restrict__ eta,
                                               const R* __restrict__ Hu, const R* __restrict__ Hv,
                                               R* Ub, R* Vb, R* dE, R* paccE, R* paccU, R* paccV,
                                               double* accE, double* accU, double* accV, R* gxe,
                                               R* gye) {
    const GeoD& g = p.g;
    if (c >= (long)g.nx * g.ny) return;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const long c2 = ix2(g, i, j);
    Ub[c2] = Un[c2];
    Vb[c2] = Vn[c2];
    dE[c2] = R(0);
    paccE[c2] = R(0);
    paccU[c2] = R(0);
    paccV[c2] = R(0);
    acc_zero<R>(accE, c2);
    acc_zero<R>(accU, c2);
    acc_zero<R>(accV, c2);
    gxe[c2] = Hu[c2] > R(0) ? R(eta[c2] - eta[c2 - 1]) : R(0);
    gye[c2] = Hv[c2] > R(0) ? R(eta[c2] - eta[c2 - g.pitch]) : R(0);
}

template <typename R>
__global__ void k_baro_begin(KP<R> p, const R* __restrict__ Un, const R* __restrict__ Vn,
                             const double* __restrict__ eta, const R* __restrict__ Hu,
                             const R* __restrict__ Hv, R* Ub, R* Vb, R* dE, R* paccE, R* paccU,
                             R* paccV, double* accE, double* accU, double* accV, R* gxe, R* gye) {
    baro_begin_col<R>(p, (long)blockIdx.x * blockDim.x + threadIdx.x, Un, Vn, eta, Hu, Hv, Ub,
                      Vb, dE, paccE, paccU, paccV, accE, accU, accV, gxe, gye);
}

// Temporal blocking of the sub-cycle (the one-GPU form of the paper's barotropic halo as
// wide as the number of substeps): a block owns a BRX x BRY region of columns in shared
// memory, an interior plus a BS-wide halo, and advances it BS substeps per pass; each
// substep's forward-backward pair shrinks the valid region by one column on each side,
// so after BS substeps the interior is exact.  One pass reads the state once and writes
// it once instead of once per substep.  The state ping-pongs between two global buffers
// across passes (neighbouring blocks read their halos from the previous pass).
constexpr int BRX = 64, BRY = 32, BS = 6, BNT = 512, BC = BRX * BRY / BNT;
// dynamic shared memory of a region: eta, U, V planes and three per-row arrays
template <typename R> constexpr size_t baro_smem() { return (3 * BRX * BRY + 3 * BRY) * sizeof(R); }
// resident blocks per SM: in FP32 two (registers <= 64), so that one block's loads
// overlap another's substeps; the FP64 form needs more registers than that allows
template <typename R> struct BaroOcc { static constexpr int value = 2; };
template <> struct BaroOcc<double> { static constexpr int value = 1; };

// padded index of (i, j) with periodic wrap; -1 beyond a wall (a region reaches less
// than one region width beyond the domain, so the wrap is one add or subtract for any
// domain at least that wide)
__device__ __forceinline__ long wrap_ix(const GeoD& g, int i, int j, int& jw) {
    if (g.px) {
        while (i < 0) i += g.nx;
        while (i >= g.nx) i -= g.nx;
    } else if (i < 0 || i >= g.nx) {
        return -1;
    }
    if (g.py) {
        while (j < 0) j += g.ny;
        while (j >= g.ny) j -= g.ny;
    } else if (j < 0 || j >= g.ny) {
        return -1;
    }
    jw = j;
    return ix2(g, i, j);
}

// region (bx, by): the interior [bx IX, bx IX + IX) x [by IY, by IY + IY) and its halo.
// WEIGHTED: the partial sums take substep m with the filter's weight fw[m] (the pass's own
// weights), else with weight 1 (equal weights, scaled by 1/N_s at the end)
template <typename R, bool WEIGHTED = false>
__device__ __forceinline__ void baro_region(
    const KP<R>& p, const int bx, const int by, const R* __restrict__ Ea,
    const R* __restrict__ Ua, const R* __restrict__ Va, R* __restrict__ Eb, R* __restrict__ Ub,
    R* __restrict__ Vb, const R* __restrict__ gxe, const R* __restrict__ gye,
    const R* __restrict__ Hu, const R* __restrict__ Hv, const R* __restrict__ GU,
    const R* __restrict__ GV, const R* __restrict__ Un, const R* __restrict__ Vn,
    double* __restrict__ accE, double* __restrict__ accU, double* __restrict__ accV, int nsub,
    R dtau, R grav, const int bs, const R* __restrict__ fw = nullptr) {
    extern __shared__ __align__(16) unsigned char bsm[];
    R* sE = reinterpret_cast<R*>(bsm);
    R* sU = sE + BRX * BRY;
    R* sV = sU + BRX * BRY;
    R* sDN = sV + BRX * BRY;   // per region row: dxv of the north and south faces and
    R* sDS = sDN + BRY;        // dtau / A_c (0 for rows outside the domain)
    R* sCe = sDS + BRY;
    const GeoD& g = p.g;
    const int tid = threadIdx.x;
    const int IX = BRX - 2 * bs, IY = BRY - 2 * bs;   // interior; the halo is bs >= nsub wide
    const int i0 = bx * IX - bs, j0 = by * IY - bs;   // region origin
    // a thread owns the cells (rx, ry0 + r), r < BC, of one region column: consecutive
    // rows, so the state of its inner cells' north and south neighbours is in its own
    // registers; shared memory carries what the neighbouring threads read
    const int rx = tid % BRX, ry0 = (tid / BRX) * BC;
    if (tid < BRY) {
        int j = j0 + tid;
        if (g.py) { j %= g.ny; if (j < 0) j += g.ny; }
        const bool in = j >= 0 && j < g.ny;
        sDS[tid] = in ? p.dxv[j + OC_H] : R(0);
        sDN[tid] = in ? p.dxv[j + 1 + OC_H] : R(0);
        sCe[tid] = in ? dtau * p.rAc[j + OC_H] : R(0);
    }
    R Au[BC], Bu[BC], Av[BC], Bv[BC], u0[BC], v0[BC];
    R pE[BC], pU[BC], pV[BC];
    R e[BC], uu[BC], vv[BC];   // the thread's own state
    unsigned wetm = 0, ownm = 0;
#pragma unroll
    for (int r = 0; r < BC; ++r) {
        const int ry = ry0 + r, q = ry * BRX + rx;
        int jw = 0;
        const long c = wrap_ix(g, i0 + rx, j0 + ry, jw);
        const bool own = rx >= bs && rx < BRX - bs && ry >= bs && ry < BRY - bs &&
                         i0 + rx < g.nx && j0 + ry < g.ny;
        ownm |= (own ? 1u : 0u) << r;
        pE[r] = pU[r] = pV[r] = R(0);
        if (c >= 0) {
            // every load of the cell issued at once (none waits on another's value)
            const R hu = Hu[c], hv = Hv[c];
            const R gu = GU[c], gv = GV[c], gx = gxe[c], gy = gye[c], rdx = p.rdxc[jw + OC_H];
            const int kbc = g.kb[c];
            e[r] = Ea[c];
            uu[r] = Ua[c];
            vv[r] = Va[c];
            u0[r] = Un[c];   // used by owned cells only
            v0[r] = Vn[c];
            // U += dtau [-g H_u (gxe + deta_i - deta_{i-1})/dx_c + G_U]
            //    = U + Bu - Au (deta_i - deta_{i-1})
            Au[r] = hu > R(0) ? dtau * grav * hu * rdx : R(0);
            Bu[r] = hu > R(0) ? dtau * gu - Au[r] * gx : R(0);
            Av[r] = hv > R(0) ? dtau * grav * hv * p.rdy : R(0);
            Bv[r] = hv > R(0) ? dtau * gv - Av[r] * gy : R(0);
            wetm |= (kbc < g.nz ? 1u : 0u) << r;
        } else {
            e[r] = uu[r] = vv[r] = R(0);
            Au[r] = Bu[r] = Av[r] = Bv[r] = u0[r] = v0[r] = R(0);
        }
        sE[q] = e[r];
        sU[q] = uu[r];
        sV[q] = vv[r];
    }
    __syncthreads();
    for (int m = 0; m < nsub; ++m) {
        const R wm = WEIGHTED ? fw[m] : R(1);
        // deta^m = deta^{m-1} - dtau/A_c [dy (U_{i+1} - U_i) + dxv_{j+1} V_{j+1} - dxv_j V_j]
        // (the east and north neighbours' U, V are read before anyone rewrites them)
#pragma unroll
        for (int r = 0; r < BC; ++r) {
            const int ry = ry0 + r, q = ry * BRX + rx;
            if (rx + 1 < BRX && ry + 1 < BRY && ((wetm >> r) & 1u)) {
                const R vN = r + 1 < BC ? vv[r + 1] : sV[q + BRX];
                const R div = p.dy * (sU[q + 1] - uu[r]) + sDN[ry] * vN - sDS[ry] * vv[r];
                e[r] = e[r] - sCe[ry] * div;
                sE[q] = e[r];
                if (WEIGHTED) pE[r] = fma(wm, e[r], pE[r]);
                else pE[r] += e[r];
            }
        }
        __syncthreads();
        // U^m, V^m from eta^m (the west and south neighbours' eta from the pass above)
#pragma unroll
        for (int r = 0; r < BC; ++r) {
            const int ry = ry0 + r, q = ry * BRX + rx;
            if (rx >= 1 && Au[r] != R(0)) {
                const R un = uu[r] + Bu[r] - Au[r] * (e[r] - sE[q - 1]);
                uu[r] = un;
                sU[q] = un;
                if (WEIGHTED) pU[r] = fma(wm, un - u0[r], pU[r]);
                else pU[r] += un - u0[r];
            }
            if (ry >= 1 && Av[r] != R(0)) {
                const R eS = r > 0 ? e[r - 1] : sE[q - BRX];
                const R vn = vv[r] + Bv[r] - Av[r] * (e[r] - eS);
                vv[r] = vn;
                if (r == 0) sV[q] = vn;   // only the thread below reads it
                if (WEIGHTED) pV[r] = fma(wm, vn - v0[r], pV[r]);
                else pV[r] += vn - v0[r];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < BC; ++r) {
        if (!((ownm >> r) & 1u)) continue;
        const int ry = ry0 + r;
        int jw = 0;
        const long c = wrap_ix(g, i0 + rx, j0 + ry, jw);
        Eb[c] = e[r];
        Ub[c] = uu[r];
        Vb[c] = vv[r];
        // one thread owns each cell: a reduction in memory is the plain FP64 add, issued
        // without waiting for the old value
        acc_add(accE, c, pE[r]);
        acc_add(accU, c, pU[r]);
        acc_add(accV, c, pV[r]);
    }
}

template <typename R, bool WEIGHTED>
__global__ void __launch_bounds__(BNT, BaroOcc<R>::value) k_baro_pass(
    KP<R> p, const R* __restrict__ Ea, const R* __restrict__ Ua, const R* __restrict__ Va,
    R* __restrict__ Eb, R* __restrict__ Ub, R* __restrict__ Vb, const R* __restrict__ gxe,
    const R* __restrict__ gye, const R* __restrict__ Hu, const R* __restrict__ Hv,
    const R* __restrict__ GU, const R* __restrict__ GV, const R* __restrict__ Un,
    const R* __restrict__ Vn, double* __restrict__ accE, double* __restrict__ accU,
    double* __restrict__ accV, int nsub, R dtau, R grav, const R* __restrict__ fw) {
    baro_region<R, WEIGHTED>(p, blockIdx.x, blockIdx.y, Ea, Ua, Va, Eb, Ub, Vb, gxe, gye, Hu, Hv,
                             GU, GV, Un, Vn, accE, accU, accV, nsub, dtau, grav, BS, fw);
}

// eta^{n+1} = eta^n + sum_m a_m deta^m in FP64; correction of the depth-integrated
// velocity (Ubar - sum dz u**)/H_u with Ubar = U^n + sum_m a_m (U^m - U^n); `rns` scales
// the accumulated sums (1/N_s for equal weights, 1 when the passes applied the weights)
template <typename R>
__device__ __forceinline__ void baro_end_col(const KP<R>& p, const long c, double* eta,
                                             const double* __restrict__ accE,
                                             const double* __restrict__ accU,
                                             const double* __restrict__ accV,
                                             const R* __restrict__ Un, const R* __restrict__ Vn,
                                             const R* __restrict__ Su, const R* __restrict__ Sv,
                                             const R* __restrict__ rHu, const R* __restrict__ rHv,
                                             R* corrU, R* corrV, double rns) {
    const GeoD& g = p.g;
    if (c >= (long)g.nx * g.ny) return;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const long c2 = ix2(g, i, j);
    if (g.kb[c2] < g.nz) eta[c2] = eta[c2] + (double)acc_scaled<R>(accE, c2, rns);
    corrU[c2] = rHu[c2] > R(0) ? (acc_scaled<R>(accU, c2, rns) + (Un[c2] - Su[c2])) * rHu[c2] : R(0);
    corrV[c2] = rHv[c2] > R(0) ? (acc_scaled<R>(accV, c2, rns) + (Vn[c2] - Sv[c2])) * rHv[c2] : R(0);
}

template <typename R>
__global__ void k_baro_end(KP<R> p, double* eta, const double* __restrict__ accE,
                           const double* __restrict__ accU, const double* __restrict__ accV,
                           const R* __restrict__ Un, const R* __restrict__ Vn,
                           const R* __restrict__ Su, const R* __restrict__ Sv,
                           const R* __restrict__ rHu, const R* __restrict__ rHv, R* corrU,
                           R* corrV, double rns) {
    baro_end_col<R>(p, (long)blockIdx.x * blockDim.x + threadIdx.x, eta, accE, accU, accV, Un,
                    Vn, Su, Sv, rHu, rHv, corrU, corrV, rns);
}

// The correction is a read-modify-write of u and v over the whole water column, split
// into slabs of CORR_SLAB levels (one slab for the usual column depths: thinner slabs
// measured slower at 1/12 degree, each re-reading the column's masks and corrections).
constexpr int CORR_SLAB = 64;

template <typename R>
__device__ __forceinline__ void correct_col(const KP<R>& p, const long c, const int slab,
                                            R* __restrict__ un, R* __restrict__ vn,
                                            const R* __restrict__ corrU,
                                            const R* __restrict__ corrV) {
    const GeoD& g = p.g;
    if (c >= (long)g.nx * g.ny) return;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const long c2 = ix2(g, i, j), P = g.plane;
    const int k0 = slab * CORR_SLAB, k1 = k0 + CORR_SLAB < g.nz ? k0 + CORR_SLAB : g.nz;
    const int ku = g.kbu[c2], kv = g.kbv[c2];
    const R cu = corrU[c2], cv = corrV[c2];
    // u and v of four levels loaded at once (eight loads in flight per column), every
    // lane of the warp on the same levels (coalesced)
    const int kmn = __reduce_min_sync(__activemask(), ku < kv ? ku : kv);
    for (int k = k0 > kmn ? k0 : kmn; k < k1; k += 4) {
        R uq[4], vq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long ck = (long)(k + q) * P + c2;
            uq[q] = k + q < k1 && k + q >= ku ? un[ck] : R(0);
            vq[q] = k + q < k1 && k + q >= kv ? vn[ck] : R(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long ck = (long)(k + q) * P + c2;
            if (k + q < k1 && k + q >= ku) un[ck] = uq[q] + cu;
            if (k + q < k1 && k + q >= kv) vn[ck] = vq[q] + cv;
        }
    }
}

template <typename R>
__global__ void k_correct(KP<R> p, R* __restrict__ un, R* __restrict__ vn,
                          const R* __restrict__ corrU, const R* __restrict__ corrV) {
    correct_col<R>(p, (long)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y, un, vn, corrU,
                   corrV);
}

// ------------------------------------------------------------------ halos

}  // namespace

// ------------------------------------------------------------------ launchers


template <typename R>
void launch_diag(const KP<R>& p, const StepBuffers<R>& b, cudaStream_t s) {
    const long n = (long)(p.g.nx + 2) * (p.g.ny + 2);
    k_diag<R><<<nblocks(n, TPB), TPB, 0, s>>>(p, b.u, b.v, b.T, b.S, b.w, b.p, b.kap, b.nu);
}

template <typename R>
void launch_tracer(const KP<R>& p, const StepBuffers<R>& b, bool step, cudaStream_t s) {
    const dim3 grid((p.g.nx + TX - 1) / TX, (p.g.ny + TY - 1) / TY), block(TX, TTY);
    const TracerArgs<R> a = tracer_args(b);
    auto go = [&](auto kern) { kern<<<grid, block, 0, s>>>(p, b.tm, a); };
    if (p.vweno) {
        if (step) go(k_tracer<R, true, true>);
        else go(k_tracer<R, false, true>);
    } else {
        if (step) go(k_tracer<R, true, false>);
        else go(k_tracer<R, false, false>);
    }
}

template <typename R>
void launch_momentum(const KP<R>& p, const StepBuffers<R>& b, bool step, cudaStream_t s) {
    const dim3 grid((p.g.nx + TX - 1) / TX, (p.g.ny + TY - 1) / TY), block(TX, TY);
    const MomentumArgs<R> a = momentum_args(b);
    auto go = [&](auto kern) { kern<<<grid, block, 0, s>>>(p, b.tm, a); };
    if (p.mvadv) {
        if (step) go(k_momentum<R, true, true>);
        else go(k_momentum<R, false, true>);
    } else {
        if (step) go(k_momentum<R, true, false>);
        else go(k_momentum<R, false, false>);
    }
}

template <typename R>
void launch_barotropic(const KP<R>& p, const StepBuffers<R>& b, int ns, double dt, R grav,
                       cudaStream_t s) {
    const GeoD& g = p.g;
    const long n = (long)g.nx * g.ny;
    const int nbk = nblocks(n, TPB);
    const R dtau = b.fw ? (R)(dt / b.fmom) : (R)(2.0 * dt / (ns + 1.0));
    if (g.px || g.py) launch_halo2<double>(g, b.eta, s);
    k_baro_begin<R><<<nbk, TPB, 0, s>>>(p, b.Un, b.Vn, b.eta, b.Hu, b.Hv, b.Ub, b.Vb, b.dE,
                                       b.paccE, b.paccU, b.paccV, b.accE, b.accU, b.accV, b.gxe,
                                       b.gye);
    const dim3 grid((g.nx + BRX - 2 * BS - 1) / (BRX - 2 * BS),
                    (g.ny + BRY - 2 * BS - 1) / (BRY - 2 * BS));
    const size_t smem = baro_smem<R>();
    R *Ea = b.dE, *Ua = b.Ub, *Va = b.Vb, *Eb = b.dE2, *Ub = b.Ub2, *Vb = b.Vb2;
    for (int m0 = 0; m0 < ns; m0 += BS) {
        const int nsub = ns - m0 < BS ? ns - m0 : BS;
        if (b.fw)
            k_baro_pass<R, true><<<grid, BNT, smem, s>>>(p, Ea, Ua, Va, Eb, Ub, Vb, b.gxe, b.gye,
                                                         b.Hu, b.Hv, b.GU, b.GV, b.Un, b.Vn,
                                                         b.accE, b.accU, b.accV, nsub, dtau,
                                                         grav, b.fw + m0);
        else
            k_baro_pass<R, false><<<grid, BNT, smem, s>>>(p, Ea, Ua, Va, Eb, Ub, Vb, b.gxe, b.gye,
                                                          b.Hu, b.Hv, b.GU, b.GV, b.Un, b.Vn,
                                                          b.accE, b.accU, b.accV, nsub, dtau,
                                                          grav, nullptr);
        R* t;
        t = Ea; Ea = Eb; Eb = t;
        t = Ua; Ua = Ub; Ub = t;
        t = Va; Va = Vb; Vb = t;
    }
    k_baro_end<R><<<nbk, TPB, 0, s>>>(p, b.eta, b.accE, b.accU, b.accV, b.Un, b.Vn, b.Su, b.Sv,
                                     b.rHu, b.rHv, b.corrU, b.corrV, b.fw ? 1.0 : 1.0 / ns);
}

int baro_passes(int ns) { return (ns + BS - 1) / BS; }

// The averaging weights.  Equal weights: a_m = 1/ns.  Power law: the shape
// s(x) = x^2 (1 - x^4) - r x, r = 0.284 (Shchepetkin & McWilliams 2005), whose support
// ends at xs, the root of x - x^5 = r beyond the maximum of x - x^5 at 5^(-1/4); Newton's
// iteration from x = 1 (where x - x^5 - r < 0 and the function is concave and falling)
// converges monotonically to it.  Sampled at m xs/(ns + 1), normalised to sum 1.
double baro_filter_weights(int ns, int kind, double* a) {
    if (kind == OCEAN_FILTER_POWER_LAW) {
        const double r = 0.284;
        double x = 1.0;
        for (int it = 0; it < 60; ++it) {
            const double x4 = x * x * x * x;
            const double f = x - x4 * x - r, df = 1.0 - 5.0 * x4;
            const double nx = x - f / df;
            if (nx == x) break;
            x = nx;
        }
        double sum = 0.0;
        for (int m = 1; m <= ns; ++m) {
            const double xm = x * m / (ns + 1.0), x2 = xm * xm;
            a[m - 1] = x2 * (1.0 - x2 * x2) - r * xm;
            sum += a[m - 1];
        }
        for (int m = 0; m < ns; ++m) a[m] /= sum;
    } else {
        for (int m = 0; m < ns; ++m) a[m] = 1.0 / ns;
    }
    double mom = 0.0;
    for (int m = 1; m <= ns; ++m) mom += m * a[m - 1];
    return mom;
}

template <typename R>
void launch_correct(const KP<R>& p, const StepBuffers<R>& b, cudaStream_t s) {
    const long n = (long)p.g.nx * p.g.ny;
    const dim3 grid(nblocks(n, TPB), (p.g.nz + CORR_SLAB - 1) / CORR_SLAB);
    k_correct<R><<<grid, TPB, 0, s>>>(p, b.un, b.vn, b.corrU, b.corrV);
}

// up to four field pointers passed by value, so a halo launch needs no device table
template <typename R> struct PtrPack { R* f[4]; };

// periodic copies: x halo columns of the interior rows, then y halo rows of the full
// padded width (so the corners come out right)

// W: the host arrays' type (double, or float); the scaling is in FP64 either way, so a
// float array and the double array of the same values give the same fields
template <typename R, typename W>
__global__ void k_wind(GeoD g, const W* __restrict__ tx, const W* __restrict__ ty,
                       double scale, R* __restrict__ ox, R* __restrict__ oy) {
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (long)g.nx * g.ny) return;
    const long c2 = ix2(g, (int)(c % g.nx), (int)(c / g.nx));
    ox[c2] = tx ? (R)((double)tx[c] * scale) : R(0);
    oy[c2] = ty ? (R)((double)ty[c] * scale) : R(0);
}

template <typename R>
__global__ void k_halo_x_pack(GeoD g, PtrPack<R> pk, int nf, int nlev) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per = (long)2 * OC_H * g.ny;
    if (t >= per * nlev * nf) return;
    const int f = (int)(t / (per * nlev));
    t -= (long)f * per * nlev;
    const int k = (int)(t / per);
    t -= (long)k * per;
    const int j = (int)(t / (2 * OC_H)), h = (int)(t % (2 * OC_H));
    const int i = h < OC_H ? h - OC_H : g.nx + (h - OC_H);
    const int isrc = h < OC_H ? i + g.nx : i - g.nx;
    R* F = pk.f[f];
    F[k * g.plane + ix2(g, i, j)] = F[k * g.plane + ix2(g, isrc, j)];
}

template <typename R>
__global__ void k_halo_y_pack(GeoD g, PtrPack<R> pk, int nf, int nlev) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = g.nx + 2 * OC_H;
    const long per = (long)2 * OC_H * W;
    if (t >= per * nlev * nf) return;
    const int f = (int)(t / (per * nlev));
    t -= (long)f * per * nlev;
    const int k = (int)(t / per);
    t -= (long)k * per;
    const int h = (int)(t / W), i = (int)(t % W) - OC_H;
    const int j = h < OC_H ? h - OC_H : g.ny + (h - OC_H);
    const int jsrc = h < OC_H ? j + g.ny : j - g.ny;
    R* F = pk.f[f];
    F[k * g.plane + ix2(g, i, j)] = F[k * g.plane + ix2(g, i, jsrc)];
}

template <typename R>
static void halo_pack(const GeoD& g, R* const* f, int nf, int nlev, cudaStream_t s) {
    PtrPack<R> pk{};
    for (int q = 0; q < nf && q < 4; ++q) pk.f[q] = f[q];
    if (g.px) {
        const long n = (long)2 * OC_H * g.ny * nlev * nf;
        k_halo_x_pack<R><<<nblocks(n, 256), 256, 0, s>>>(g, pk, nf, nlev);
    }
    if (g.py) {
        const long n = (long)2 * OC_H * (g.nx + 2 * OC_H) * nlev * nf;
        k_halo_y_pack<R><<<nblocks(n, 256), 256, 0, s>>>(g, pk, nf, nlev);
    }
}

template <typename R>
void launch_halo3(const GeoD& g, R* const* f, int nf, cudaStream_t s) {
    for (int q = 0; q < nf; q += 4) halo_pack<R>(g, f + q, nf - q < 4 ? nf - q : 4, g.nz, s);
}

template <typename R, typename W>
void launch_wind(const GeoD& g, const W* tx, const W* ty, double scale, R* ox, R* oy,
                 cudaStream_t s) {
    const long n = (long)g.nx * g.ny;
    k_wind<R, W><<<nblocks(n, TPB), TPB, 0, s>>>(g, tx, ty, scale, ox, oy);
}

template <typename R>
void launch_halo2(const GeoD& g, R* f, cudaStream_t s) {
    halo_pack<R>(g, &f, 1, 1, s);
}

// ------------------------------------------------------------------ diagnostics

namespace {

// Neumaier-compensated pair (s, c)
struct CSum {
    double s, c;
};
__device__ __forceinline__ void cs_add(CSum& a, double x) {
    const double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}
__device__ __forceinline__ void cs_merge(CSum& a, const CSum& b) {
    cs_add(a, b.s);
    a.c += b.c;
}

// One column per thread: the column's T' dz, S' dz in the path's precision from its
// lowest wet level (in the mixed form an FP32 sum of at most nz terms, far below the 1e-6
// the mixed conservation holds to), plus the reference part and the volume from the
// per-kb sums, in FP64; kinetic energy and the CFL number in the state's own precision.
// The block's columns are then summed in FP64 by a pairwise tree in a fixed order (warp
// shuffles, then the eight warp sums): its rounding error is at most log2(256) units of
// FP64 roundoff of the summed magnitudes, and the cheap FP64 adds keep GB300's slow FP64
// rate off the path.  The blocks' partial sums are merged with Neumaier compensation by
// k_diag_final.
// IDX: the element index type (32-bit offsets when every field fits, fewer registers)
template <typename R, typename IDX>
__global__ void __launch_bounds__(OC_DIAG_THREADS) k_diag_sums(
    GeoD g, DiagMetrics m, const R* __restrict__ u, const R* __restrict__ v,
    const R* __restrict__ T, const R* __restrict__ S, const double* __restrict__ eta,
    double* __restrict__ partials) {
    double vT = 0.0, vS = 0.0, vE = 0.0, vK = 0.0, vV = 0.0;
    R cflr = R(0);
    bool bad = false;
    const long ncol = (long)g.nx * g.ny;
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncol) {
        const R dtr = (R)m.dt, rdyr = (R)m.rdy;
        const int i = (int)(c % g.nx), j = (int)(c / g.nx);
        const long c2 = ix2(g, i, j);
        const int kb = g.kb[c2], ku = g.kbu[c2], kv = g.kbv[c2];
        const double ac = m.Ac[j + OC_H], av = m.dxv[j + OC_H] * m.dy;
        const R rdx = (R)m.rdxc[j + OC_H];
        // w of the current state for its CFL number, integrated up from the sea floor as
        // the diagnostics kernel does (same operands and order): w = 0 on the floor,
        // w_{k+1} = w_k - rac (dy dz_k (u_{i+1} - u_i) + dz_k (dxv_{j+1} v_{j+1} - dxv_j v_j))
        const R dyr = (R)m.dy, dxvS = (R)m.dxv[j + OC_H], dxvN = (R)m.dxv[j + 1 + OC_H];
        const R rac = (R)(1.0 / m.Ac[j + OC_H]);
        R wk = R(0);
        // land cells hold 0 and are skipped
        R tcol = R(0), scol = R(0);
        R ku2 = R(0), kv2 = R(0);
        const int k0 = __reduce_min_sync(__activemask(), min(kb, min(ku, kv)));   // warp-uniform
        const IDX plane = (IDX)g.plane, pitch = (IDX)g.pitch;
        IDX ck0 = (IDX)k0 * plane + (IDX)c2;
        // four levels' operands loaded at once (24 loads in flight per column), then used
        for (int k4 = k0; k4 < g.nz; k4 += 4, ck0 += 4 * plane) {
            R tq[4], sq[4], uq[4], vq[4], ueq[4], vnq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const IDX ck = ck0 + (IDX)q * plane;
                const bool in = k4 + q < g.nz;
                tq[q] = in ? T[ck] : R(0);
                sq[q] = in ? S[ck] : R(0);
                uq[q] = in ? u[ck] : R(0);
                vq[q] = in ? v[ck] : R(0);
                ueq[q] = in ? u[ck + 1] : R(0);
                vnq[q] = in ? v[ck + pitch] : R(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k4 + q;
                if (k >= g.nz) break;
                // one test for the four values (a NaN or infinity in any makes the sum
                // non-finite; physical values are far from overflowing it)
                bad = bad || !isfinite(tq[q] + sq[q] + uq[q] + vq[q]);
                const R dzr = (R)m.dz[k];
                if (k >= kb) {
                    tcol = fma(tq[q], dzr, tcol);
                    scol = fma(sq[q], dzr, scol);
                    cflr = fmax(cflr, fabs(wk) * (R)m.dtdz[k]);   // w on the level's floor
                    if (k < g.nz - 1) {
                        const R div = dyr * dzr * (ueq[q] - uq[q]) + dzr * (dxvN * vnq[q] - dxvS * vq[q]);
                        wk = wk - div * rac;
                    }
                }
                if (k >= ku) {
                    ku2 += uq[q] * uq[q] * dzr;
                    cflr = fmax(cflr, fabs(uq[q]) * dtr * rdx);
                }
                if (k >= kv) {
                    kv2 += vq[q] * vq[q] * dzr;
                    cflr = fmax(cflr, fabs(vq[q]) * dtr * rdyr);
                }
            }
        }
        if (kb < g.nz) {
            vT = ((double)tcol + m.colT[kb]) * ac;
            vS = ((double)scol + m.colS[kb]) * ac;
            vV = m.colV[kb] * ac;
            vE = eta[c2] * ac;
        }
        vK = 0.5 * ((double)ku2 * ac + (double)kv2 * av);
        bad = bad || !isfinite(eta[c2]);
    }
    double cfl = (double)cflr;
    int nb = bad ? 1 : 0;
    // pairwise tree over the warp (lane l adds lane l + off), then over the warps
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        vT += __shfl_down_sync(0xffffffffu, vT, off);
        vS += __shfl_down_sync(0xffffffffu, vS, off);
        vE += __shfl_down_sync(0xffffffffu, vE, off);
        vK += __shfl_down_sync(0xffffffffu, vK, off);
        vV += __shfl_down_sync(0xffffffffu, vV, off);
        cfl = fmax(cfl, __shfl_down_sync(0xffffffffu, cfl, off));
        nb |= __shfl_down_sync(0xffffffffu, nb, off);
    }
    constexpr int NW = OC_DIAG_THREADS / 32;
    __shared__ double ws[7][NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        ws[0][wid] = vT; ws[1][wid] = vS; ws[2][wid] = vE; ws[3][wid] = vK; ws[4][wid] = vV;
        ws[5][wid] = cfl; ws[6][wid] = (double)nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* o = partials + (long)blockIdx.x * 12;
        for (int q = 0; q < 5; ++q) {
            double a[NW];
            for (int w = 0; w < NW; ++w) a[w] = ws[q][w];
            for (int h = NW / 2; h > 0; h >>= 1)
                for (int w = 0; w < h; ++w) a[w] += a[w + h];
            o[2 * q] = a[0];
            o[2 * q + 1] = 0.0;   // compensation term of the block sum (merged by k_diag_final)
        }
        double cm = 0.0, bm = 0.0;
        for (int w = 0; w < NW; ++w) {
            cm = fmax(cm, ws[5][w]);
            bm = fmax(bm, ws[6][w]);
        }
        o[10] = cm;
        o[11] = bm;
    }
}

// The mixed form of the same reduction without FP64 arithmetic per cell (GB300's FP64
// unit runs conversions and adds at a small fraction of the FP32 rate, and the FP64
// reduction spent most of its time there): the metrics come as FP32 copies, each
// column's anomaly content and kinetic energy are formed in FP32 and summed over the warp
// by the same pairwise tree in FP32, and only then widened, per warp, into the block's
// FP64 tree.  The reference profiles' part of the tracer totals and the wet volume do
// not change with the state: the host forms them once in FP64 and the final merge adds
// them.  sum eta dA stays FP64 per column (eta is the FP64 state).
template <typename IDX>
__global__ void __launch_bounds__(OC_DIAG_THREADS) k_diag_sums_f32(
    GeoD g, DiagMetrics m, const float* __restrict__ u, const float* __restrict__ v,
    const float* __restrict__ T, const float* __restrict__ S, const double* __restrict__ eta,
    double* __restrict__ partials) {
    float fT = 0.f, fS = 0.f, fK = 0.f, cflr = 0.f;
    double vE = 0.0;
    bool bad = false;
    const long ncol = (long)g.nx * g.ny;
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncol) {
        const int i = (int)(c % g.nx), j = (int)(c / g.nx), jr = j + OC_H;
        const long c2 = ix2(g, i, j);
        const int kb = g.kb[c2], ku = g.kbu[c2], kv = g.kbv[c2];
        const float ac = m.fAc[jr], av = m.fdxv[jr] * m.fdy, rdx = m.frdxc[jr];
        const float dyr = m.fdy, dxvS = m.fdxv[jr], dxvN = m.fdxv[jr + 1], rac = m.frAc[jr];
        const float dtr = m.fdt, rdyr = m.frdy;
        // w for the CFL number, integrated up from the sea floor as in the FP64 form
        float wk = 0.f, tcol = 0.f, scol = 0.f, ku2 = 0.f, kv2 = 0.f;
        const int k0 = __reduce_min_sync(__activemask(), min(kb, min(ku, kv)));   // warp-uniform
        const IDX plane = (IDX)g.plane, pitch = (IDX)g.pitch;
        IDX ck0 = (IDX)k0 * plane + (IDX)c2;
        // four levels' operands loaded at once (24 loads in flight per column), then used
        for (int k4 = k0; k4 < g.nz; k4 += 4, ck0 += 4 * plane) {
            float tq[4], sq[4], uq[4], vq[4], ueq[4], vnq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const IDX ck = ck0 + (IDX)q * plane;
                const bool in = k4 + q < g.nz;
                tq[q] = in ? T[ck] : 0.f;
                sq[q] = in ? S[ck] : 0.f;
                uq[q] = in ? u[ck] : 0.f;
                vq[q] = in ? v[ck] : 0.f;
                ueq[q] = in ? u[ck + 1] : 0.f;
                vnq[q] = in ? v[ck + pitch] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k4 + q;
                if (k >= g.nz) break;
                bad = bad || !isfinite(tq[q] + sq[q] + uq[q] + vq[q]);
                const float dzr = m.fdz[k];
                if (k >= kb) {
                    tcol = fmaf(tq[q], dzr, tcol);
                    scol = fmaf(sq[q], dzr, scol);
                    cflr = fmaxf(cflr, fabsf(wk) * m.fdtdz[k]);   // w on the level's floor
                    if (k < g.nz - 1) {
                        const float div = dyr * dzr * (ueq[q] - uq[q]) + dzr * (dxvN * vnq[q] - dxvS * vq[q]);
                        wk = wk - div * rac;
                    }
                }
                if (k >= ku) {
                    ku2 += uq[q] * uq[q] * dzr;
                    cflr = fmaxf(cflr, fabsf(uq[q]) * dtr * rdx);
                }
                if (k >= kv) {
                    kv2 += vq[q] * vq[q] * dzr;
                    cflr = fmaxf(cflr, fabsf(vq[q]) * dtr * rdyr);
                }
            }
        }
        if (kb < g.nz) {
            fT = tcol * ac;
            fS = scol * ac;
            vE = eta[c2] * m.Ac[jr];
        }
        fK = 0.5f * (ku2 * ac + kv2 * av);
        bad = bad || !isfinite(eta[c2]);
    }
    int nb = bad ? 1 : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        fT += __shfl_down_sync(0xffffffffu, fT, off);
        fS += __shfl_down_sync(0xffffffffu, fS, off);
        fK += __shfl_down_sync(0xffffffffu, fK, off);
        vE += __shfl_down_sync(0xffffffffu, vE, off);
        cflr = fmaxf(cflr, __shfl_down_sync(0xffffffffu, cflr, off));
        nb |= __shfl_down_sync(0xffffffffu, nb, off);
    }
    constexpr int NW = OC_DIAG_THREADS / 32;
    __shared__ double ws[7][NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        ws[0][wid] = (double)fT; ws[1][wid] = (double)fS; ws[2][wid] = vE; ws[3][wid] = (double)fK;
        ws[4][wid] = 0.0;   // the wet volume is a constant of the grid (added at the end)
        ws[5][wid] = (double)cflr; ws[6][wid] = (double)nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* o = partials + (long)blockIdx.x * 12;
        for (int q = 0; q < 5; ++q) {
            double a[NW];
            for (int w = 0; w < NW; ++w) a[w] = ws[q][w];
            for (int h = NW / 2; h > 0; h >>= 1)
                for (int w = 0; w < h; ++w) a[w] += a[w + h];
            o[2 * q] = a[0];
            o[2 * q + 1] = 0.0;
        }
        double cm = 0.0, bm = 0.0;
        for (int w = 0; w < NW; ++w) {
            cm = fmax(cm, ws[5][w]);
            bm = fmax(bm, ws[6][w]);
        }
        o[10] = cm;
        o[11] = bm;
    }
}

// One block merges FIN_TH consecutive partials (of the first nblk) into partial blockIdx.x
// of `merged`, with compensation, in a fixed tree: the FP64 work of the merge spread over
// the GPU instead of one SM.
constexpr int FIN_TH = 256;
__global__ void __launch_bounds__(FIN_TH) k_diag_merge(const double* __restrict__ partials,
                                                       int nblk, double* __restrict__ merged) {
    __shared__ CSum red[5][FIN_TH];
    __shared__ double rc[FIN_TH], rb[FIN_TH];
    const int t = threadIdx.x;
    const long b = (long)blockIdx.x * FIN_TH + t;
    for (int q = 0; q < 5; ++q) red[q][t] = CSum{0, 0};
    rc[t] = 0.0;
    rb[t] = 0.0;
    if (b < nblk) {
        const double* o = partials + b * 12;
        for (int q = 0; q < 5; ++q) red[q][t] = CSum{o[2 * q], o[2 * q + 1]};
        rc[t] = o[10];
        rb[t] = o[11];
    }
    __syncthreads();
    for (int h = FIN_TH / 2; h > 0; h >>= 1) {
        if (t < h) {
            for (int q = 0; q < 5; ++q) cs_merge(red[q][t], red[q][t + h]);
            rc[t] = fmax(rc[t], rc[t + h]);
            rb[t] = fmax(rb[t], rb[t + h]);
        }
        __syncthreads();
    }
    if (t == 0) {
        double* o = merged + (long)blockIdx.x * 12;
        for (int q = 0; q < 5; ++q) { o[2 * q] = red[q][0].s; o[2 * q + 1] = red[q][0].c; }
        o[10] = rc[0];
        o[11] = rb[0];
    }
}

// the per-block partial sums merged in a fixed tree: each of 256 threads merges
// nblk / 256 consecutive partials, then pairs of threads halve the set
__global__ void __launch_bounds__(FIN_TH) k_diag_final(const double* __restrict__ partials,
                                                       int nblk, double* out, double cT,
                                                       double cS, double cV) {
    __shared__ CSum red[5][FIN_TH];
    __shared__ double rc[FIN_TH], rb[FIN_TH];
    const int t = threadIdx.x;
    CSum a[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    double cfl = 0.0, bad = 0.0;
    for (int b = t; b < nblk; b += FIN_TH) {
        const double* o = partials + (long)b * 12;
        for (int q = 0; q < 5; ++q) cs_merge(a[q], CSum{o[2 * q], o[2 * q + 1]});
        cfl = fmax(cfl, o[10]);
        bad = fmax(bad, o[11]);
    }
    for (int q = 0; q < 5; ++q) red[q][t] = a[q];
    rc[t] = cfl;
    rb[t] = bad;
    __syncthreads();
    for (int h = FIN_TH / 2; h > 0; h >>= 1) {
        if (t < h) {
            for (int q = 0; q < 5; ++q) cs_merge(red[q][t], red[q][t + h]);
            rc[t] = fmax(rc[t], rc[t + h]);
            rb[t] = fmax(rb[t], rb[t + h]);
        }
        __syncthreads();
    }
    if (t == 0) {
        // cT, cS, cV: the reference part of the totals when the blocks summed anomalies
        // only (the mixed form), else 0
        out[0] = cT + (red[0][0].s + red[0][0].c);
        out[1] = cS + (red[1][0].s + red[1][0].c);
        out[2] = red[2][0].s + red[2][0].c;
        out[3] = red[3][0].s + red[3][0].c;
        out[4] = rc[0];
        out[5] = rb[0];
        out[6] = cV + (red[4][0].s + red[4][0].c);
        out[7] = 0.0;
    }
}

}  // namespace

size_t diag_partials_bytes(long ncol) {
    const long nblk = (ncol + OC_DIAG_THREADS - 1) / OC_DIAG_THREADS;
    const long nmrg = (nblk + FIN_TH - 1) / FIN_TH;
    return (size_t)(nblk + nmrg) * 12 * sizeof(double);
}

template <typename R>
void launch_diagnostics(const GeoD& g, const DiagMetrics& m, const R* u, const R* v, const R* T,
                        const R* S, const double* eta, double* partials, double* out,
                        cudaStream_t s) {
    const long ncol = (long)g.nx * g.ny;
    const int nblk = (int)((ncol + OC_DIAG_THREADS - 1) / OC_DIAG_THREADS);
    const bool small = (unsigned long long)g.plane * g.nz < (1ull << 32);
    if constexpr (sizeof(R) == sizeof(float)) {
        if (small)
            k_diag_sums_f32<unsigned><<<nblk, OC_DIAG_THREADS, 0, s>>>(g, m, u, v, T, S, eta, partials);
        else
            k_diag_sums_f32<long><<<nblk, OC_DIAG_THREADS, 0, s>>>(g, m, u, v, T, S, eta, partials);
    } else if (small) {
        k_diag_sums<R, unsigned><<<nblk, OC_DIAG_THREADS, 0, s>>>(g, m, u, v, T, S, eta, partials);
    } else {
        k_diag_sums<R, long><<<nblk, OC_DIAG_THREADS, 0, s>>>(g, m, u, v, T, S, eta, partials);
    }
    // the block partials merged by blocks of FIN_TH, then those by one block
    const int nmrg = (nblk + FIN_TH - 1) / FIN_TH;
    double* merged = partials + (long)nblk * 12;
    k_diag_merge<<<nmrg, FIN_TH, 0, s>>>(partials, nblk, merged);
    const bool f32 = sizeof(R) == sizeof(float);
    k_diag_final<<<1, FIN_TH, 0, s>>>(merged, nmrg, out, f32 ? m.cT : 0.0, f32 ? m.cS : 0.0,
                                      f32 ? m.cV : 0.0);
}

// ------------------------------------------------------------------ batched ensemble
// Persistent kernels over a work list of (member, position) items.  A block takes items
// blockIdx.x, blockIdx.x + gridDim.x, ... (static schedule) or the next item of an
// atomic counter (dynamic schedule); the host sorts the list by decreasing cost, so
// either schedule hands out the long items first.  Each item runs the same body as the
// single-model kernel, with the member's parameters and buffers from a device table.

namespace {

__device__ __forceinline__ int ens_first(int* counter, int* s_next) {
    if (!counter) return blockIdx.x;
    if (threadIdx.x == 0 && threadIdx.y == 0) *s_next = atomicAdd(counter, 1);
    __syncthreads();
    return *s_next;
}

// the barrier frees the item's shared memory (and *s_next) for the next item
__device__ __forceinline__ int ens_next(int* counter, int* s_next, int it) {
    __syncthreads();
    if (!counter) return it + gridDim.x;
    if (threadIdx.x == 0 && threadIdx.y == 0) *s_next = atomicAdd(counter, 1);
    __syncthreads();
    return *s_next;
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_ens_diag(const EnsMember<R>* __restrict__ mem,
                                                  const EnsItem* __restrict__ work, int nwork,
                                                  int* counter) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const KP<R>& p = mem[e.m].k;
        const StepBuffers<R>& b = mem[e.m].b;
        diag_col<R>(p, (long)e.a * TPB + threadIdx.x, b.u, b.v, b.T, b.S, b.w, b.p, b.kap, b.nu);
    }
}

template <typename R>
__global__ void __launch_bounds__(NTT, (OccX<R, true>::value)) k_ens_tracer(
    const EnsMember<R>* __restrict__ mem, const EnsItem* __restrict__ work, int nwork,
    int* counter) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const StepBuffers<R>& b = mem[e.m].b;
        tracer_tile<R, true, false, long>(mem[e.m].k, b.tm, e.a, e.b, tracer_args(b));
    }
}

template <typename R>
__global__ void __launch_bounds__(NT, (OccX<R, true>::value)) k_ens_momentum(
    const EnsMember<R>* __restrict__ mem, const EnsItem* __restrict__ work, int nwork,
    int* counter) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const StepBuffers<R>& b = mem[e.m].b;
        momentum_tile<R, true, false, long>(mem[e.m].k, b.tm, e.a, e.b, momentum_args(b));
    }
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_ens_baro_begin(const EnsMember<R>* __restrict__ mem,
                                                        const EnsItem* __restrict__ work,
                                                        int nwork, int* counter) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const KP<R>& p = mem[e.m].k;
        const StepBuffers<R>& b = mem[e.m].b;
        baro_begin_col<R>(p, (long)e.a * TPB + threadIdx.x, b.Un, b.Vn, b.eta, b.Hu, b.Hv, b.Ub,
                          b.Vb, b.dE, b.paccE, b.paccU, b.paccV, b.accE, b.accU, b.accV, b.gxe,
                          b.gye);
    }
}

// odd passes run from the second buffers back into the first, as in the single model
template <typename R>
__global__ void __launch_bounds__(BNT, BaroOcc<R>::value) k_ens_baro_pass(const EnsMember<R>* __restrict__ mem,
                                                       const EnsItem* __restrict__ work,
                                                       int nwork, int* counter, int odd,
                                                       int nsub, int bs) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const KP<R>& p = mem[e.m].k;
        const StepBuffers<R>& b = mem[e.m].b;
        const R dtau = mem[e.m].dtau;
        R *Ea = b.dE, *Ua = b.Ub, *Va = b.Vb, *Eb = b.dE2, *Ub = b.Ub2, *Vb = b.Vb2;
        if (odd) {
            Ea = b.dE2; Ua = b.Ub2; Va = b.Vb2;
            Eb = b.dE; Ub = b.Ub; Vb = b.Vb;
        }
        baro_region<R>(p, e.a, e.b, Ea, Ua, Va, Eb, Ub, Vb, b.gxe, b.gye, b.Hu, b.Hv, b.GU, b.GV,
                       b.Un, b.Vn, b.accE, b.accU, b.accV, nsub, dtau, p.grav, bs);
    }
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_ens_baro_end(const EnsMember<R>* __restrict__ mem,
                                                      const EnsItem* __restrict__ work,
                                                      int nwork, int* counter) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const KP<R>& p = mem[e.m].k;
        const StepBuffers<R>& b = mem[e.m].b;
        baro_end_col<R>(p, (long)e.a * TPB + threadIdx.x, b.eta, b.accE, b.accU, b.accV, b.Un,
                        b.Vn, b.Su, b.Sv, b.rHu, b.rHv, b.corrU, b.corrV, mem[e.m].rns);
    }
}

template <typename R>
__global__ void __launch_bounds__(TPB) k_ens_correct(const EnsMember<R>* __restrict__ mem,
                                                     const EnsItem* __restrict__ work,
                                                     int nwork, int* counter) {
    __shared__ int s_next;
    for (int it = ens_first(counter, &s_next); it < nwork; it = ens_next(counter, &s_next, it)) {
        const EnsItem e = work[it];
        const KP<R>& p = mem[e.m].k;
        const StepBuffers<R>& b = mem[e.m].b;
        correct_col<R>(p, (long)e.a * TPB + threadIdx.x, e.b, b.un, b.vn, b.corrU, b.corrV);
    }
}

}  // namespace

EnsShape ens_shape() { return EnsShape{TPB, TX, TY, BRX, BRY, BS, CORR_SLAB}; }

template <typename R>
int ens_blocks_per_sm(int kind) {
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (kind) {
        case ENS_DIAG: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_diag<R>, TPB, 0); break;
        case ENS_TRACER: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_tracer<R>, NTT, 0); break;
        case ENS_MOMENTUM: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_momentum<R>, NT, 0); break;
        case ENS_BARO_BEGIN: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_baro_begin<R>, TPB, 0); break;
        case ENS_BARO_PASS:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_baro_pass<R>, BNT,
                                                              baro_smem<R>());
            break;
        case ENS_BARO_END: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_baro_end<R>, TPB, 0); break;
        case ENS_CORRECT: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_correct<R>, TPB, 0); break;
        default: return 0;
    }
    return e == cudaSuccess ? n : 0;
}

template <typename R>
void launch_ens(int kind, const EnsMember<R>* mem, const EnsItem* work, int nwork, int grid,
                int* counter, int odd, int nsub, int bs, cudaStream_t s) {
    if (nwork <= 0 || grid <= 0) return;
    const dim3 tile(TX, TY);
    switch (kind) {
        case ENS_DIAG: k_ens_diag<R><<<grid, TPB, 0, s>>>(mem, work, nwork, counter); break;
        case ENS_TRACER: k_ens_tracer<R><<<grid, dim3(TX, TTY), 0, s>>>(mem, work, nwork, counter); break;
        case ENS_MOMENTUM: k_ens_momentum<R><<<grid, tile, 0, s>>>(mem, work, nwork, counter); break;
        case ENS_BARO_BEGIN: k_ens_baro_begin<R><<<grid, TPB, 0, s>>>(mem, work, nwork, counter); break;
        case ENS_BARO_PASS:
            k_ens_baro_pass<R><<<grid, BNT, baro_smem<R>(), s>>>(
                mem, work, nwork, counter, odd, nsub, bs);
            break;
        case ENS_BARO_END: k_ens_baro_end<R><<<grid, TPB, 0, s>>>(mem, work, nwork, counter); break;
        case ENS_CORRECT: k_ens_correct<R><<<grid, TPB, 0, s>>>(mem, work, nwork, counter); break;
        default: break;
    }
}

// the FP64 region (three planes and the row arrays) is just above the 48 KB of dynamic
// shared memory a kernel gets without opting in
template <typename R>
int setup_kernel_attributes(int nz) {
    (void)nz;
    const int bytes = (int)baro_smem<R>();
    cudaError_t e = cudaFuncSetAttribute(k_baro_pass<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_baro_pass<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ens_baro_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return (int)e;
}

// 1 if a tile kernel's bounded wait gave up since the last call (the flag is cleared)
int tile_wait_failed() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tile_err, sizeof(int)) != cudaSuccess) return 1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tile_err, &z, sizeof(int));
    }
    return v;
}

// ------------------------------------------------------------------ instantiations

#define OC_INST(R)                                                                          \
    template int setup_kernel_attributes<R>(int);                                           \
    template void launch_diag<R>(const KP<R>&, const StepBuffers<R>&, cudaStream_t);        \
    template void launch_tracer<R>(const KP<R>&, const StepBuffers<R>&, bool, cudaStream_t); \
    template void launch_momentum<R>(const KP<R>&, const StepBuffers<R>&, bool,             \
                                     cudaStream_t);                                         \
    template void launch_barotropic<R>(const KP<R>&, const StepBuffers<R>&, int, double, R, \
                                       cudaStream_t);                                       \
    template void launch_correct<R>(const KP<R>&, const StepBuffers<R>&, cudaStream_t);     \
    template void launch_halo3<R>(const GeoD&, R* const*, int, cudaStream_t);               \
    template void launch_halo2<R>(const GeoD&, R*, cudaStream_t);                           \
    template void launch_wind<R, double>(const GeoD&, const double*, const double*, double, \
                                         R*, R*, cudaStream_t);                             \
    template void launch_wind<R, float>(const GeoD&, const float*, const float*, double, R*, \
                                        R*, cudaStream_t);                                  \
    template void launch_diagnostics<R>(const GeoD&, const DiagMetrics&, const R*, const R*, \
                                        const R*, const R*, const double*, double*, double*, \
                                        cudaStream_t);                \
    template int ens_blocks_per_sm<R>(int);                                                 \
    template void launch_ens<R>(int, const EnsMember<R>*, const EnsItem*, int, int, int*,   \
                                int, int, int, cudaStream_t);

OC_INST(double)
OC_INST(float)
