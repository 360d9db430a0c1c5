// ocean_closure.cu -- model-side kernels of the learned column closure: network inputs
// from a model state, the network outputs applied inside the step (a diffusivity added
// to the Richardson-number one and tracer-tendency corrections, neither applied to a
// column whose outputs are not finite), and the training targets obtained by coarse-graining
// a fine model onto a coarse one (r x r blocks of columns, same levels).
#include <cuda_bf16.h>

#include "ocean_internal.cuh"

namespace {

constexpr int CT = 128;
inline int cblocks(long n) { return (int)((n + CT - 1) / CT); }

__device__ __forceinline__ float softplus_c(float z) { return z > 20.f ? z : log1pf(__expf(z)); }

// Per interior column c = j nx + i: raw features (T, S, centre u, v on levels; N^2 and
// shear^2 on bottom faces), z-scored with mu and 1/sigma where the entry counts (wet level or
// interior face), else 0, for the levels [k0, k1).  emit(fi, x, k, w, f, gT, gS) receives
// feature fi = q nz + k, its value, and for q = 0 the level's masks and vertical
// gradients.
template <typename R, typename Emit>
__device__ __forceinline__ void column_features(const KP<R>& p, long c, int k0, int k1,
                                                const R* __restrict__ u,
                                                const R* __restrict__ v, const R* __restrict__ T,
                                                const R* __restrict__ S,
                                                const float* __restrict__ mu,
                                                const float* __restrict__ rsigma, Emit emit) {
    const GeoD& g = p.g;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx), nz = g.nz;
    const long c2 = ix2(g, i, j), P = g.plane;
    const int kb = g.kb[c2];
    float ubp = 0.f, vbp = 0.f;   // centre u, v of level k-1 (0 below the sea floor)
    if (k0 > 0 && k0 - 1 >= kb) {
        const long cm = (long)(k0 - 1) * P + c2;
        ubp = 0.5f * (float)(u[cm] + u[cm + 1]);
        vbp = 0.5f * (float)(v[cm] + v[cm + g.pitch]);
    }
    for (int k = k0; k < k1; ++k) {
        const long ck = k * P + c2;
        const bool w = k >= kb, f = k >= kb + 1;
        const float ub = w ? 0.5f * (float)(u[ck] + u[ck + 1]) : 0.f;
        const float vb = w ? 0.5f * (float)(v[ck] + v[ck + g.pitch]) : 0.f;
        float n2 = 0.f, sh2 = 0.f, gT = 0.f, gS = 0.f;
        if (f) {
            const float rz = (float)p.rdzf[k];
            gT = (float)((T[ck] - T[ck - P]) + p.dTref[k]) * rz;
            gS = (float)((S[ck] - S[ck - P]) + p.dSref[k]) * rz;
            n2 = (float)p.grav * ((float)p.alpha * gT - (float)p.beta_s * gS);
            sh2 = ((ub - ubp) * (ub - ubp) + (vb - vbp) * (vb - vbp)) * rz * rz;
        }
        ubp = ub;
        vbp = vb;
        // T and S are stored as anomalies from the level reference, which is close to
        // the feature mean: (T' + (Tref - mu)) keeps the resolution (T - mu) would lose.
        // In FP32 the difference Tref - mu is exact when the two lie within a factor of
        // two of each other (Sterbenz), so one rounding of the sum gives what the FP64 sum
        // rounded to FP32 gives; otherwise one more FP32 rounding, far below the BF16
        // rounding of the feature.  No FP64 arithmetic (GB300's FP64 rate is a small
        // fraction of its FP32 rate)
        float cT = 0.f, cS = 0.f;
        if (w) {
            if constexpr (sizeof(R) == sizeof(float)) {
                cT = (float)T[ck] + ((float)p.Tref[k] - mu[k]);
                cS = (float)S[ck] + ((float)p.Sref[k] - mu[nz + k]);
            } else {
                cT = (float)((double)T[ck] + ((double)p.Tref[k] - (double)mu[k]));
                cS = (float)((double)S[ck] + ((double)p.Sref[k] - (double)mu[nz + k]));
            }
        }
        const float raw[6] = {cT, cS, ub - mu[2 * nz + k], vb - mu[3 * nz + k],
                              n2 - mu[4 * nz + k], sh2 - mu[5 * nz + k]};
        const bool use[6] = {w, w, w, w, f, f};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int fi = q * nz + k;
            emit(fi, use[q] ? raw[q] * rsigma[fi] : 0.f, k, w, f, gT, gS);
        }
    }
}

// features, masks and gradients of every column, one thread per column (the training
// pipeline's extraction)
template <typename R>
__global__ void k_closure_features(KP<R> p, const R* __restrict__ u, const R* __restrict__ v,
                                   const R* __restrict__ T, const R* __restrict__ S,
                                   const float* __restrict__ mu, const float* __restrict__ rsigma,
                                   float* __restrict__ Xf, __nv_bfloat16* __restrict__ Xb,
                                   unsigned char* __restrict__ face, unsigned char* __restrict__ wet,
                                   float* __restrict__ dzT, float* __restrict__ dzS) {
    const GeoD& g = p.g;
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (long)g.nx * g.ny) return;
    const int nz = g.nz;
    column_features<R>(p, c, 0, nz, u, v, T, S, mu, rsigma,
                       [&](int fi, float x, int k, bool w, bool f, float gT, float gS) {
                           if (Xf) Xf[c * 6 * nz + fi] = x;
                           if (Xb) Xb[c * 6 * nz + fi] = __float2bfloat16_rn(x);
                           if (fi == k) {
                               if (face) face[c * nz + k] = f;
                               if (wet) wet[c * nz + k] = w;
                               if (dzT) dzT[c * nz + k] = gT;
                               if (dzS) dzS[c * nz + k] = gS;
                           }
                       });
}

// Rows of feature matrices and network outputs pass through shared memory, so the
// row-major [column][feature] arrays are written and read with coalesced accesses
// (one thread per column would touch one 2- or 4-byte element per row per access).  A
// block of 32 columns x XQ level ranges: thread (c, q) handles the levels
// [q L, q L + L) of column c, L = ceil(nz / XQ), so that a column's serial chain of
// loads is an eighth as long; rows padded by one 4-byte word (no bank conflicts).
constexpr int XC = 32, XQ = 8;

// BF16 features of the step's network pass (no masks or gradients)
template <typename R>
__global__ void __launch_bounds__(XC * XQ) k_closure_xb(KP<R> p, const R* __restrict__ u,
                                                        const R* __restrict__ v,
                                                        const R* __restrict__ T,
                                                        const R* __restrict__ S,
                                                        const float* __restrict__ mu,
                                                        const float* __restrict__ rsigma,
                                                        __nv_bfloat16* __restrict__ Xb) {
    extern __shared__ __align__(16) unsigned char fx_raw[];
    __nv_bfloat16* tile = reinterpret_cast<__nv_bfloat16*>(fx_raw);
    const GeoD& g = p.g;
    const int nz = g.nz, F = 6 * nz, ld = F + 2;
    const long ncol = (long)g.nx * g.ny, c0 = (long)blockIdx.x * XC;
    const int t = threadIdx.x, tc = t % XC, tq = t / XC;
    const int L = (nz + XQ - 1) / XQ, k0 = tq * L, k1 = min(k0 + L, nz);
    if (c0 + tc < ncol && k0 < k1) {
        __nv_bfloat16* row = tile + (long)tc * ld;
        column_features<R>(p, c0 + tc, k0, k1, u, v, T, S, mu, rsigma,
                           [&](int fi, float x, int, bool, bool, float, float) {
                               row[fi] = __float2bfloat16_rn(x);
                           });
    }
    __syncthreads();
    // the block's rows are contiguous in Xb: copy them out as 4-byte pairs (F is even)
    const long rows = ncol - c0 < XC ? ncol - c0 : XC;
    const int pairs = F / 2;
    unsigned* dst = reinterpret_cast<unsigned*>(Xb + c0 * F);
    for (long q = t; q < rows * pairs; q += blockDim.x) {
        const long r = q / pairs, e = q - r * pairs;
        dst[q] = *reinterpret_cast<const unsigned*>(tile + r * ld + 2 * e);
    }
}

// network outputs -> extra diffusivity on the interior wet faces (added to the
// Richardson-number value already in kap) and tracer corrections; the block's rows of Y
// come in through shared memory (coalesced), each column's levels split as above
template <typename R>
__global__ void __launch_bounds__(XC * XQ) k_closure_apply(KP<R> p, const float* __restrict__ Y,
                                                           float ks, float gt, float gs,
                                                           R* __restrict__ kap,
                                                           R* __restrict__ dGT,
                                                           R* __restrict__ dGS) {
    extern __shared__ __align__(16) unsigned char fy_raw[];
    float* tile = reinterpret_cast<float*>(fy_raw);
    __shared__ int s_ok[XC];
    const GeoD& g = p.g;
    const int nz = g.nz, F = 3 * nz, ld = F + 1;
    const long ncol = (long)g.nx * g.ny, c0 = (long)blockIdx.x * XC;
    const int t = threadIdx.x, tc = t % XC, tq = t / XC;
    const long rows = ncol - c0 < XC ? ncol - c0 : XC;
    const float* src = Y + c0 * F;
    for (long q = t; q < rows * F; q += blockDim.x) {
        const long r = q / F;
        tile[r * ld + (q - r * F)] = src[q];
    }
    __syncthreads();
    if (tq == 0) {   // a column's outputs are applied only if all of them are finite
        bool ok = true;
        const float* y = tile + (long)tc * ld;
        for (int q = 0; q < F; ++q) ok = ok && isfinite(y[q]);
        s_ok[tc] = ok ? 1 : 0;
    }
    __syncthreads();
    const int L = (nz + XQ - 1) / XQ, k0 = tq * L, k1 = min(k0 + L, nz);
    if (c0 + tc >= ncol || k0 >= k1) return;
    const long c = c0 + tc;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const long c2 = ix2(g, i, j), P = g.plane;
    const int kb = g.kb[c2];
    const float* y = tile + (long)tc * ld;
    const bool ok = s_ok[tc] != 0;
    for (int k = k0; k < k1; ++k) {
        const long ck = k * P + c2;
        if (ok && k >= kb + 1) kap[ck] = kap[ck] + (R)(ks * softplus_c(y[k]));
        dGT[ck] = (ok && k >= kb) ? (R)(gt * y[nz + k]) : R(0);
        dGS[ck] = (ok && k >= kb) ? (R)(gs * y[2 * nz + k]) : R(0);
    }
}

// Coarse-grain a fine model onto a coarse one (r x r columns per coarse column):
// tracer anomalies and fine tendencies as volume-weighted means over the wet fine cells,
// u, v as means over the wet fine faces lying on the coarse face, eta as the area-
// weighted mean over wet fine columns; subgrid vertical fluxes <w T_f> - <w><T_f> over
// the wet fine faces (T_f the mean of the two cells around the face).  Dry coarse
// entries get 0.  Both models use the same reference profiles, so anomalies average.
template <typename R>
__global__ void k_coarse_grain(KP<R> pf, KP<R> pc, int r, const R* __restrict__ uf,
                               const R* __restrict__ vf, const R* __restrict__ Tf,
                               const R* __restrict__ Sf, const R* __restrict__ wf,
                               const R* __restrict__ GTf, const R* __restrict__ GSf,
                               const double* __restrict__ etaf, R* __restrict__ uc,
                               R* __restrict__ vc, R* __restrict__ Tc, R* __restrict__ Sc,
                               double* __restrict__ etac, float* __restrict__ FT,
                               float* __restrict__ FS, float* __restrict__ GTm,
                               float* __restrict__ GSm) {
    const GeoD& gf = pf.g;
    const GeoD& gc = pc.g;
    const long C = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= (long)gc.nx * gc.ny) return;
    const int I = (int)(C % gc.nx), J = (int)(C / gc.nx), nz = gc.nz;
    const long C2 = ix2(gc, I, J), Pc = gc.plane, Pf = gf.plane;
    const int kbc = gc.kb[C2], kbuc = gc.kbu[C2], kbvc = gc.kbv[C2];
    // free surface
    double se = 0.0, sa = 0.0;
    for (int b = 0; b < r; ++b) {
        const int jf = r * J + b;
        const double area = 1.0 / (double)pf.rAc[jf + OC_H];
        for (int a = 0; a < r; ++a) {
            const long c2 = ix2(gf, r * I + a, jf);
            if (gf.kb[c2] < nz) {
                se += etaf[c2] * area;
                sa += area;
            }
        }
    }
    etac[C2] = (kbc < nz && sa > 0.0) ? se / sa : 0.0;
    for (int k = 0; k < nz; ++k) {
        double sT = 0, sS = 0, sw = 0, sgT = 0, sgS = 0;
        double fw = 0, fTf = 0, fSf = 0, fwT = 0, fwS = 0, fa = 0;
        for (int b = 0; b < r; ++b) {
            const int jf = r * J + b;
            const double area = 1.0 / (double)pf.rAc[jf + OC_H];
            for (int a = 0; a < r; ++a) {
                const long c2 = ix2(gf, r * I + a, jf), ck = k * Pf + c2;
                const int kb = gf.kb[c2];
                if (k >= kb) {
                    sT += (double)Tf[ck] * area;
                    sS += (double)Sf[ck] * area;
                    sgT += (double)GTf[ck] * area;
                    sgS += (double)GSf[ck] * area;
                    sw += area;
                }
                if (k >= kb + 1) {
                    const double w = (double)wf[ck];
                    const double tfc = 0.5 * ((double)Tf[ck] + (double)Tf[ck - Pf]);
                    const double sfc = 0.5 * ((double)Sf[ck] + (double)Sf[ck - Pf]);
                    fw += w * area;
                    fTf += tfc * area;
                    fSf += sfc * area;
                    fwT += w * tfc * area;
                    fwS += w * sfc * area;
                    fa += area;
                }
            }
        }
        const long Ck = k * Pc + C2;
        const bool cw = k >= kbc;
        Tc[Ck] = (cw && sw > 0) ? (R)(sT / sw) : R(0);
        Sc[Ck] = (cw && sw > 0) ? (R)(sS / sw) : R(0);
        GTm[C * nz + k] = (cw && sw > 0) ? (float)(sgT / sw) : 0.f;
        GSm[C * nz + k] = (cw && sw > 0) ? (float)(sgS / sw) : 0.f;
        const bool cf = k >= kbc + 1 && fa > 0;
        FT[C * nz + k] = cf ? (float)(fwT / fa - (fw / fa) * (fTf / fa)) : 0.f;
        FS[C * nz + k] = cf ? (float)(fwS / fa - (fw / fa) * (fSf / fa)) : 0.f;
        // u on the coarse west face: fine faces (rI, rJ + b)
        double su = 0;
        int nu = 0;
        for (int b = 0; b < r; ++b) {
            const long c2 = ix2(gf, r * I, r * J + b);
            if (k >= gf.kbu[c2]) {
                su += (double)uf[k * Pf + c2];
                ++nu;
            }
        }
        uc[Ck] = (k >= kbuc && nu > 0) ? (R)(su / nu) : R(0);
        double sv = 0;
        int nv = 0;
        for (int a = 0; a < r; ++a) {
            const long c2 = ix2(gf, r * I + a, r * J);
            if (k >= gf.kbv[c2]) {
                sv += (double)vf[k * Pf + c2];
                ++nv;
            }
        }
        vc[Ck] = (k >= kbvc && nv > 0) ? (R)(sv / nv) : R(0);
    }
}

// lateral residual target: <G_fine> - G_coarse + (F_{k+1} - F_k)/dz_k on wet coarse levels
template <typename R>
__global__ void k_closure_targets(KP<R> p, const R* __restrict__ GcT, const R* __restrict__ GcS,
                                  const float* __restrict__ GTm, const float* __restrict__ GSm,
                                  const float* __restrict__ FT, const float* __restrict__ FS,
                                  float* __restrict__ GTt, float* __restrict__ GSt) {
    const GeoD& g = p.g;
    const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (long)g.nx * g.ny) return;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx), nz = g.nz;
    const long c2 = ix2(g, i, j), P = g.plane;
    const int kb = g.kb[c2];
    for (int k = 0; k < nz; ++k) {
        const long q = c * nz + k;
        if (k < kb) {
            GTt[q] = 0.f;
            GSt[q] = 0.f;
            continue;
        }
        const float ftu = k + 1 < nz ? FT[q + 1] : 0.f, fsu = k + 1 < nz ? FS[q + 1] : 0.f;
        const float rdz = (float)p.rdz[k];
        GTt[q] = GTm[q] - (float)GcT[k * P + c2] + (ftu - FT[q]) * rdz;
        GSt[q] = GSm[q] - (float)GcS[k * P + c2] + (fsu - FS[q]) * rdz;
    }
}

}  // namespace

template <typename R>
void launch_closure_features(const KP<R>& p, const R* u, const R* v, const R* T, const R* S,
                             const float* mu, const float* rsigma, float* Xf, void* Xb,
                             unsigned char* face, unsigned char* wet, float* dzT, float* dzS,
                             cudaStream_t s) {
    const long ncol = (long)p.g.nx * p.g.ny;
    if (Xb && !Xf && !face && !wet && !dzT && !dzS) {   // the step's BF16 features
        const size_t smem = (size_t)XC * (6 * p.g.nz + 2) * sizeof(__nv_bfloat16);
        k_closure_xb<R><<<(int)((ncol + XC - 1) / XC), XC * XQ, smem, s>>>(
            p, u, v, T, S, mu, rsigma, reinterpret_cast<__nv_bfloat16*>(Xb));
        return;
    }
    k_closure_features<R><<<cblocks(ncol), CT, 0, s>>>(
        p, u, v, T, S, mu, rsigma, Xf, reinterpret_cast<__nv_bfloat16*>(Xb), face, wet, dzT, dzS);
}

template <typename R>
void launch_closure_apply(const KP<R>& p, const float* Y, float ks, float gt, float gs, R* kap,
                          R* dGT, R* dGS, cudaStream_t s) {
    const long ncol = (long)p.g.nx * p.g.ny;
    const size_t smem = (size_t)XC * (3 * p.g.nz + 1) * sizeof(float);
    k_closure_apply<R><<<(int)((ncol + XC - 1) / XC), XC * XQ, smem, s>>>(p, Y, ks, gt, gs, kap,
                                                                          dGT, dGS);
}

// the tiled kernels' shared memory (above the default 48 KB for nz > 125); set before the
// first launch and outside stream capture
template <typename R>
int closure_tiles_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_closure_xb<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         100 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_closure_apply<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 100 * 1024);
    return (int)e;
}

template <typename R>
void launch_coarse_grain(const KP<R>& pf, const KP<R>& pc, int r, const R* uf, const R* vf,
                         const R* Tf, const R* Sf, const R* wf, const R* GTf, const R* GSf,
                         const double* etaf, R* uc, R* vc, R* Tc, R* Sc, double* etac, float* FT,
                         float* FS, float* GTm, float* GSm, cudaStream_t s) {
    k_coarse_grain<R><<<cblocks((long)pc.g.nx * pc.g.ny), CT, 0, s>>>(
        pf, pc, r, uf, vf, Tf, Sf, wf, GTf, GSf, etaf, uc, vc, Tc, Sc, etac, FT, FS, GTm, GSm);
}

template <typename R>
void launch_closure_targets(const KP<R>& p, const R* GcT, const R* GcS, const float* GTm,
                            const float* GSm, const float* FT, const float* FS, float* GTt,
                            float* GSt, cudaStream_t s) {
    k_closure_targets<R><<<cblocks((long)p.g.nx * p.g.ny), CT, 0, s>>>(p, GcT, GcS, GTm, GSm, FT,
                                                                        FS, GTt, GSt);
}

#define OC_CLOSURE_INST(R)                                                                      \
    template void launch_closure_features<R>(const KP<R>&, const R*, const R*, const R*,       \
                                             const R*, const float*, const float*, float*,     \
                                             void*, unsigned char*, unsigned char*, float*,    \
                                             float*, cudaStream_t);                            \
    template int closure_tiles_setup<R>();                                                     \
    template void launch_closure_apply<R>(const KP<R>&, const float*, float, float, float, R*, \
                                          R*, R*, cudaStream_t);                               \
    template void launch_coarse_grain<R>(const KP<R>&, const KP<R>&, int, const R*, const R*,  \
                                         const R*, const R*, const R*, const R*, const R*,     \
                                         const double*, R*, R*, R*, R*, double*, float*,       \
                                         float*, float*, float*, cudaStream_t);                \
    template void launch_closure_targets<R>(const KP<R>&, const R*, const R*, const float*,    \
                                            const float*, const float*, const float*, float*,  \
                                            float*, cudaStream_t);

OC_CLOSURE_INST(double)
OC_CLOSURE_INST(float)
