// ocean_internal.cuh -- device-side layout, kernel parameters and shared device
// functions of the GB300 ocean step.  Included by the kernel and host translation units
// of libocean only.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ocean.h"

// Horizontal halo width of every padded field: five-point WENO stencils reach three
// cells beyond a face, staggered averages one more.
#define OC_H 4
// Columns of one block of the 2.5-D tracer and momentum tiles (x by y); the host's tensor
// maps use the same numbers for their boxes.
#define OC_TX 32
#define OC_TY 8
// Largest number of levels the column kernels accept.
#define OC_NZMAX 192

// Geometry and masks shared by all kernels.  Padded 2-D index of column (i, j):
// (j + OC_H) * pitch + (i + OC_H), for i in [-OC_H, nx + OC_H), j in [-OC_H, ny + OC_H).
// 3-D index: k * plane + that.
struct GeoD {
    int nx, ny, nz, px, py, pitch;
    long plane;
    const short* kb;     // lowest wet level of each column (nz = land)
    const short* kbu;    // lowest wet level of the u-face on the west side of the column
    const short* kbv;    // lowest wet level of the v-face on the south side
    const short* kbz;    // corner (SW of the column) active, all four cells wet, for k >= kbz
    const short* kbzin;  // corner touches the fluid (one cell wet) for k >= kbzin
};

__device__ __forceinline__ long ix2(const GeoD& g, int i, int j) {
    return (long)(j + OC_H) * g.pitch + (i + OC_H);
}

// Metrics, constants and switches passed by value to every kernel.  R is the storage
// and arithmetic type of the 3-D fields (double, or float in the mixed form).
template <typename R>
struct KP {
    GeoD g;
    // per-row metrics, indexed j + OC_H
    const R *dxc, *rdxc, *dxv, *rAc, *rAz, *fu, *fv;
    // per-level metrics: dz[k], 1/dz[k], dzf[k] = zc[k] - zc[k-1], 1/dzf[k]; the
    // horizontally uniform reference profiles Tref, Sref (T and S are stored as anomalies
    // T - Tref(k), S - Sref(k)) and their level differences dTref[k] = Tref[k] - Tref[k-1]
    const R *dz, *rdz, *dzf, *rdzf, *Tref, *Sref, *dTref, *dSref;
    R dy, rdy, dt, ca, cb;
    R grav, alpha, beta_s;
    R nu0, ri_a, nu_b, kappa_b, kappa_conv;
    R eps, ptop;
    int linear;
    // vertical schemes: vweno = 1 takes the vertical WENO coefficients of each level face
    // from vw (rows of OC_VWROW values, row (kf * 2 + dir) for face kf = 0..nz, dir 0 when
    // the face velocity is >= 0: c[3][3], d[3], c3[2][2], d3[2], 0, 0); mvadv = 1: the WENO
    // flux form of the vertical momentum advection
    const R* vw;
    int vweno, mvadv;
    // per-level rows of OC_LVROW values (see LevelRow)
    const R* lvt;
};

// One level's constants for the tile kernels, one row of KP::lvt (OC_LVROW values):
// dz_k, 1/dz_k; the implicit solve's factors alo = dt/(dz_k dzf_k) (0 at k = 0) and
// ahi = dt/(dz_k dzf_{k+1}) (0 at the top); Tref_k, Sref_k; and the diffusion of the
// reference profiles hdT = ahi (Tref_{k+1} - Tref_k), ldT = alo (Tref_k - Tref_{k-1}),
// hdS, ldS likewise for S; the rest zero.  The kernels read each value where they use
// it (short live ranges keep the tiles free of register spills).
#define OC_LVROW 16
// values per row of KP::vw
#define OC_VWROW 20

template <typename R> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
__device__ __forceinline__ float2 make_vec2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 make_vec2(double a, double b) { return make_double2(a, b); }

// ----------------------------------------------------------------------- WENO-Z

// In FP32 the ratio tau/(beta + eps) can exceed sqrt(FLT_MAX) when a stencil is
// exactly flat; above 1e18 every stencil it is compared with is smooth to far below
// FP32 resolution, so clamping leaves the reconstructed value unchanged.
template <typename R> struct WenoRatio {
    static __device__ __forceinline__ R clamp(R r) { return r; }
};
template <> struct WenoRatio<float> {
    static __device__ __forceinline__ float clamp(float r) { return fminf(r, 1e18f); }
};

// Fifth-order WENO-Z value at the face downstream of q2 (q0..q4 upwind to downwind):
// Jiang-Shu candidates and smoothness indicators, ideal weights (1, 6, 3)/10,
// alpha_r = d_r (1 + (tau5 / (beta_r + eps))^2), tau5 = |beta_0 - beta_2|.
template <typename R>
__device__ __forceinline__ R weno5(R q0, R q1, R q2, R q3, R q4, R eps, int linear) {
    const R s6 = R(1) / R(6);
    R p0 = (R(2) * q0 - R(7) * q1 + R(11) * q2) * s6;
    R p1 = (-q1 + R(5) * q2 + R(2) * q3) * s6;
    R p2 = (R(2) * q2 + R(5) * q3 - q4) * s6;
    if (linear) return R(0.1) * p0 + R(0.6) * p1 + R(0.3) * p2;
    const R c13 = R(13) / R(12);
    R a = q0 - R(2) * q1 + q2, b = q0 - R(4) * q1 + R(3) * q2;
    R b0 = c13 * a * a + R(0.25) * b * b;
    a = q1 - R(2) * q2 + q3; b = q1 - q3;
    R b1 = c13 * a * a + R(0.25) * b * b;
    a = q2 - R(2) * q3 + q4; b = R(3) * q2 - R(4) * q3 + q4;
    R b2 = c13 * a * a + R(0.25) * b * b;
    R tau = fabs(b0 - b2);
    R r0 = WenoRatio<R>::clamp(tau / (b0 + eps));
    R r1 = WenoRatio<R>::clamp(tau / (b1 + eps));
    R r2 = WenoRatio<R>::clamp(tau / (b2 + eps));
    R a0 = R(0.1) * (R(1) + r0 * r0);
    R a1 = R(0.6) * (R(1) + r1 * r1);
    R a2 = R(0.3) * (R(1) + r2 * r2);
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

// Third-order WENO-Z at the face downstream of q1 (q0..q2 upwind to downwind).
template <typename R>
__device__ __forceinline__ R weno3(R q0, R q1, R q2, R eps, int linear) {
    R p0 = R(0.5) * (-q0 + R(3) * q1);
    R p1 = R(0.5) * (q1 + q2);
    const R d0 = R(1) / R(3), d1 = R(2) / R(3);
    if (linear) return d0 * p0 + d1 * p1;
    R b0 = (q1 - q0) * (q1 - q0);
    R b1 = (q2 - q1) * (q2 - q1);
    R tau = fabs(b0 - b1);
    R r0 = WenoRatio<R>::clamp(tau / (b0 + eps));
    R r1 = WenoRatio<R>::clamp(tau / (b1 + eps));
    R a0 = d0 * (R(1) + r0 * r0);
    R a1 = d1 * (R(1) + r1 * r1);
    return (a0 * p0 + a1 * p1) / (a0 + a1);
}

// Adaptive order: bit n of `in` says whether stencil point n lies in the fluid.  All
// five: WENO5; the central three: WENO3; otherwise the upwind value q2.
template <typename R>
__device__ __forceinline__ R weno_adaptive(const R* q, unsigned in, R eps, int linear) {
    if (in == 31u) return weno5(q[0], q[1], q[2], q[3], q[4], eps, linear);
    if ((in & 14u) == 14u) return weno3(q[1], q[2], q[3], eps, linear);
    return q[2];
}

// ----------------------------------------------------------------- stretched-level WENO
// The same reconstructions with the candidates and ideal weights of one stencil of
// stretched levels (a row of the vw table: c[r][0..2] the candidate r's weights on its
// three cells, d[r] the ideal weights, c3 and d3 those of the third-order scheme on the
// central three cells).  The smoothness indicators keep their index-space form.
template <typename R>
__device__ __forceinline__ R weno5_row(const R* q, const R* c, R eps, int linear) {
    R p0 = c[0] * q[0] + c[1] * q[1] + c[2] * q[2];
    R p1 = c[3] * q[1] + c[4] * q[2] + c[5] * q[3];
    R p2 = c[6] * q[2] + c[7] * q[3] + c[8] * q[4];
    if (linear) return c[9] * p0 + c[10] * p1 + c[11] * p2;
    const R c13 = R(13) / R(12);
    R a = q[0] - R(2) * q[1] + q[2], b = q[0] - R(4) * q[1] + R(3) * q[2];
    R b0 = c13 * a * a + R(0.25) * b * b;
    a = q[1] - R(2) * q[2] + q[3]; b = q[1] - q[3];
    R b1 = c13 * a * a + R(0.25) * b * b;
    a = q[2] - R(2) * q[3] + q[4]; b = R(3) * q[2] - R(4) * q[3] + q[4];
    R b2 = c13 * a * a + R(0.25) * b * b;
    R tau = fabs(b0 - b2);
    R r0 = WenoRatio<R>::clamp(tau / (b0 + eps));
    R r1 = WenoRatio<R>::clamp(tau / (b1 + eps));
    R r2 = WenoRatio<R>::clamp(tau / (b2 + eps));
    R a0 = c[9] * (R(1) + r0 * r0);
    R a1 = c[10] * (R(1) + r1 * r1);
    R a2 = c[11] * (R(1) + r2 * r2);
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

// third order on q[1..3]
template <typename R>
__device__ __forceinline__ R weno3_row(const R* q, const R* c, R eps, int linear) {
    R p0 = c[12] * q[1] + c[13] * q[2];
    R p1 = c[14] * q[2] + c[15] * q[3];
    if (linear) return c[16] * p0 + c[17] * p1;
    R b0 = (q[2] - q[1]) * (q[2] - q[1]);
    R b1 = (q[3] - q[2]) * (q[3] - q[2]);
    R tau = fabs(b0 - b1);
    R r0 = WenoRatio<R>::clamp(tau / (b0 + eps));
    R r1 = WenoRatio<R>::clamp(tau / (b1 + eps));
    R a0 = c[16] * (R(1) + r0 * r0);
    R a1 = c[17] * (R(1) + r1 * r1);
    return (a0 * p0 + a1 * p1) / (a0 + a1);
}

template <typename R>
__device__ __forceinline__ R weno_adaptive_row(const R* q, unsigned in, const R* c, R eps, int linear) {
    if (in == 31u) return weno5_row(q, c, eps, linear);
    if ((in & 14u) == 14u) return weno3_row(q, c, eps, linear);
    return q[2];
}

// ----------------------------------------------------------------------- paired WENO
// Two reconstructions that share one stencil and one mask (T and S on the same face, or
// the two vorticity reconstructions of a thread): in FP32 they run as one stream of
// Blackwell's packed two-lane FP32 instructions (fma/mul/add .f32x2), with the weights'
// divisions as fast reciprocals; in FP64 as two scalar calls.

template <typename R> struct WenoPair {
    static __device__ __forceinline__ void run(const R* qa, const R* qb, unsigned ina,
                                               unsigned inb, R eps, int linear, R& oa, R& ob) {
        oa = weno_adaptive(qa, ina, eps, linear);
        ob = weno_adaptive(qb, inb, eps, linear);
    }
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// approximate reciprocal of the special-function unit (rcp.approx)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}

// fifth-order WENO-Z of two stencils at once (same definition as weno5, rearranged in
// first differences D_n = q_{n+1} - q_n):
//   second differences A_r = D_{r+1} - D_r; B_0 = A_0 + 2 D_1, B_1 = -(D_1 + D_2),
//   B_2 = A_2 - 2 D_2, with 4 beta_r = (13/3) A_r^2 + B_r^2, so tau5/(beta_r + eps) =
//   4 (beta_0 - beta_2) / (4 beta_r + 4 eps) needs no division by 4;
//   the candidates as 6 p_r = 6 q_2 + delta_r, delta_0 = 3 D_1 + 2 A_0,
//   delta_1 = 2 D_2 + D_1, delta_2 = 3 D_2 - A_2;
//   the value q_2 + sum_r alpha_r delta_r / (6 sum_r alpha_r).
// tau/(beta+eps) squared is clamped at 1e36 (see WenoRatio: the clamp leaves the value
// unchanged) so that the weights stay finite.
__device__ __forceinline__ float2 weno5z_x2(float2 q0, float2 q1, float2 q2, float2 q3,
                                            float2 q4, float eps) {
    const float2 D0 = f2sub(q1, q0), D1 = f2sub(q2, q1), D2 = f2sub(q3, q2), D3 = f2sub(q4, q3);
    const float2 A0 = f2sub(D1, D0), A1 = f2sub(D2, D1), A2 = f2sub(D3, D2);
    const float2 B0 = f2fma(D1, f2(2.f), A0);
    const float2 E1 = f2add(D1, D2);                 // -B_1
    const float2 B2 = f2fma(D2, f2(-2.f), A2);
    const float2 c = f2(13.f / 3.f);
    const float2 b0 = f2fma(f2mul(A0, A0), c, f2mul(B0, B0));
    const float2 b1 = f2fma(f2mul(A1, A1), c, f2mul(E1, E1));
    const float2 b2 = f2fma(f2mul(A2, A2), c, f2mul(B2, B2));
    const float2 d = f2sub(b0, b2);
    const float2 e4 = f2(4.f * eps);
    auto alpha = [&](float2 b, float dr) {
        const float2 be = f2add(b, e4);
        const float2 r = f2mul(d, make_float2(rcp_approx(be.x), rcp_approx(be.y)));
        float2 r2 = f2mul(r, r);
        r2.x = fminf(r2.x, 1e36f);
        r2.y = fminf(r2.y, 1e36f);
        return f2fma(r2, f2(dr), f2(dr));
    };
    const float2 a0 = alpha(b0, 0.1f), a1 = alpha(b1, 0.6f), a2 = alpha(b2, 0.3f);
    const float2 t3 = f2(3.f);
    const float2 g0 = f2fma(D1, t3, f2add(A0, A0));
    const float2 g1 = f2add(E1, D2);
    const float2 g2 = f2sub(f2mul(D2, t3), A2);
    const float2 num = f2fma(a0, g0, f2fma(a1, g1, f2mul(a2, g2)));
    const float2 den = f2mul(f2add(f2add(a0, a1), a2), f2(6.f));
    return f2fma(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)), q2);
}

// third-order WENO-Z of two stencils at once (same definition as weno3)
__device__ __forceinline__ float2 weno3z_x2(float2 q0, float2 q1, float2 q2, float eps) {
    const float2 h = f2(0.5f);
    const float2 p0 = f2mul(f2fma(q1, f2(3.f), f2mul(q0, f2(-1.f))), h);
    const float2 p1 = f2mul(f2add(q1, q2), h);
    const float2 e0 = f2fma(q0, f2(-1.f), q1), e1 = f2fma(q1, f2(-1.f), q2);
    const float2 b0 = f2mul(e0, e0), b1 = f2mul(e1, e1);
    const float2 tau = make_float2(fabsf(b0.x - b1.x), fabsf(b0.y - b1.y));
    const float2 r0 = make_float2(fminf(__fdividef(tau.x, b0.x + eps), 1e18f),
                                  fminf(__fdividef(tau.y, b0.y + eps), 1e18f));
    const float2 r1 = make_float2(fminf(__fdividef(tau.x, b1.x + eps), 1e18f),
                                  fminf(__fdividef(tau.y, b1.y + eps), 1e18f));
    const float2 a0 = f2mul(f2(1.f / 3.f), f2fma(r0, r0, f2(1.f)));
    const float2 a1 = f2mul(f2(2.f / 3.f), f2fma(r1, r1, f2(1.f)));
    const float2 num = f2fma(a0, p0, f2mul(a1, p1));
    const float2 den = f2add(a0, a1);
    return make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
}

// FP32: every order of the adaptive scheme in packed form.  Both stencils complete:
// one WENO5 pass.  Otherwise each of the two takes its own order (WENO5, WENO3 or the
// upwind value) from at most one WENO5 and one WENO3 pass over both, so that a warp
// whose lanes mix orders runs each pass once.
template <> struct WenoPair<float> {
    static __device__ __forceinline__ void run(const float* qa, const float* qb, unsigned ina,
                                               unsigned inb, float eps, int linear, float& oa,
                                               float& ob) {
        if (linear) {
            oa = weno_adaptive(qa, ina, eps, linear);
            ob = weno_adaptive(qb, inb, eps, linear);
            return;
        }
        const bool a5 = ina == 31u, b5 = inb == 31u;
        if (a5 && b5) {
            const float2 o = weno5z_x2(make_float2(qa[0], qb[0]), make_float2(qa[1], qb[1]),
                                       make_float2(qa[2], qb[2]), make_float2(qa[3], qb[3]),
                                       make_float2(qa[4], qb[4]), eps);
            oa = o.x;
            ob = o.y;
            return;
        }
        const bool a3 = !a5 && (ina & 14u) == 14u, b3 = !b5 && (inb & 14u) == 14u;
        oa = qa[2];
        ob = qb[2];
        if (a5 || b5) {
            const float2 o = weno5z_x2(make_float2(qa[0], qb[0]), make_float2(qa[1], qb[1]),
                                       make_float2(qa[2], qb[2]), make_float2(qa[3], qb[3]),
                                       make_float2(qa[4], qb[4]), eps);
            if (a5) oa = o.x;
            if (b5) ob = o.y;
        }
        if (a3 || b3) {
            const float2 o = weno3z_x2(make_float2(qa[1], qb[1]), make_float2(qa[2], qb[2]),
                                       make_float2(qa[3], qb[3]), eps);
            if (a3) oa = o.x;
            if (b3) ob = o.y;
        }
    }
};

// Stretched-level pairs: stencil a with table row ca, stencil b with row cb (the two
// rows may differ, e.g. u- and v-faces with opposite vertical velocities).
template <typename R> struct WenoPairRow {
    static __device__ __forceinline__ void run(const R* qa, const R* qb, unsigned ina,
                                               unsigned inb, const R* ca, const R* cb, R eps,
                                               int linear, R& oa, R& ob) {
        oa = weno_adaptive_row(qa, ina, ca, eps, linear);
        ob = weno_adaptive_row(qb, inb, cb, eps, linear);
    }
};

__device__ __forceinline__ float2 ldrow2(const float* ca, const float* cb, int n) {
    return make_float2(__ldg(ca + n), __ldg(cb + n));
}

// packed fifth-order WENO-Z with per-lane rows (same definition as weno5_row); the
// indicators are formed as in weno5z_x2 (4 beta_r, no division by 4)
__device__ __forceinline__ float2 weno5z_x2_row(float2 q0, float2 q1, float2 q2, float2 q3,
                                                float2 q4, const float* ca, const float* cb,
                                                float eps) {
    const float2 P0 = f2fma(q0, ldrow2(ca, cb, 0), f2fma(q1, ldrow2(ca, cb, 1), f2mul(q2, ldrow2(ca, cb, 2))));
    const float2 P1 = f2fma(q1, ldrow2(ca, cb, 3), f2fma(q2, ldrow2(ca, cb, 4), f2mul(q3, ldrow2(ca, cb, 5))));
    const float2 P2 = f2fma(q2, ldrow2(ca, cb, 6), f2fma(q3, ldrow2(ca, cb, 7), f2mul(q4, ldrow2(ca, cb, 8))));
    const float2 A0 = f2add(f2fma(q1, f2(-2.f), q0), q2);
    const float2 A1 = f2add(f2fma(q2, f2(-2.f), q1), q3);
    const float2 A2 = f2add(f2fma(q3, f2(-2.f), q2), q4);
    const float2 B0 = f2fma(f2fma(q1, f2(-1.f), q2), f2(2.f), A0);
    const float2 B1 = f2fma(q3, f2(-1.f), q1);
    const float2 B2 = f2fma(f2fma(q3, f2(-1.f), q2), f2(2.f), A2);
    const float2 c = f2(13.f / 3.f);
    const float2 b0 = f2fma(f2mul(A0, A0), c, f2mul(B0, B0));
    const float2 b1 = f2fma(f2mul(A1, A1), c, f2mul(B1, B1));
    const float2 b2 = f2fma(f2mul(A2, A2), c, f2mul(B2, B2));
    const float2 d = f2fma(b2, f2(-1.f), b0);
    const float2 e4 = f2(4.f * eps);
    auto alpha = [&](float2 b, float2 dr) {
        const float2 be = f2add(b, e4);
        const float2 r = f2mul(d, make_float2(rcp_approx(be.x), rcp_approx(be.y)));
        float2 r2 = f2mul(r, r);
        r2.x = fminf(r2.x, 1e36f);
        r2.y = fminf(r2.y, 1e36f);
        return f2fma(r2, dr, dr);
    };
    const float2 a0 = alpha(b0, ldrow2(ca, cb, 9)), a1 = alpha(b1, ldrow2(ca, cb, 10)),
                 a2 = alpha(b2, ldrow2(ca, cb, 11));
    const float2 num = f2fma(a0, P0, f2fma(a1, P1, f2mul(a2, P2)));
    const float2 den = f2add(f2add(a0, a1), a2);
    return f2mul(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
}

template <> struct WenoPairRow<float> {
    static __device__ __forceinline__ void run(const float* qa, const float* qb, unsigned ina,
                                               unsigned inb, const float* ca, const float* cb,
                                               float eps, int linear, float& oa, float& ob) {
        const bool a5 = ina == 31u, b5 = inb == 31u;
        if (linear || !(a5 || b5)) {   // ideal weights, or neither stencil complete
            oa = weno_adaptive_row(qa, ina, ca, eps, linear);
            ob = weno_adaptive_row(qb, inb, cb, eps, linear);
            return;
        }
        const float2 o = weno5z_x2_row(make_float2(qa[0], qb[0]), make_float2(qa[1], qb[1]),
                                       make_float2(qa[2], qb[2]), make_float2(qa[3], qb[3]),
                                       make_float2(qa[4], qb[4]), ca, cb, eps);
        oa = a5 ? o.x : weno_adaptive_row(qa, ina, ca, eps, linear);
        ob = b5 ? o.y : weno_adaptive_row(qb, inb, cb, eps, linear);
    }
};

// ----------------------------------------------------------------------- launchers
// Implemented in ocean_kernels.cu, instantiated for double and float.

// Tensor maps (TMA descriptors) of the fields the tile kernels stage, for one buffer
// parity: 3-D [nz][ny + 2H][pitch] views, one level per copy.  Tracer: T and S (boxes of
// 40 x 14 columns x rows), u and v faces (36 x 8, 32 x 9), and its own columns' w,
// diffusivity, G_T and G_S (32 x 8).  Momentum: u (40 x 14), v (40 x 13), pressure, w and
// nu (36 x 9), and its own columns' G_u and G_v (32 x 8).
struct __align__(128) TileMaps {
    CUtensorMap T, S, tu, tv, tw, tk, tgt, tgs, mu, mv, mp, mw, mnu, mgu, mgv;
};

// Encodes a tiled tensor map through the driver's entry point; false if refused.
bool oc_encode_tiled(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* ptr,
                     const unsigned long long* dims, const unsigned long long* strides,
                     const unsigned* box, CUtensorMapSwizzle swizzle);

template <typename R> struct StepBuffers {
    // state n (read) and n+1 (written)
    const R *u, *v, *T, *S;
    R *un, *vn, *Tn, *Sn;
    R *Gu, *Gv, *GT, *GS;      // G^{n-1} in, G^n out
    R *w, *p, *kap, *nu;       // diagnostics (kap also holds the tracers' Thomas c')
    R *wk;                     // 3-D scratch (the v-viscosity Thomas c')
    const R *dGT, *dGS;        // learned-closure tracer tendency corrections (or null)
    const R *taux_s, *tauy_s;  // wind stress / (rho0 dz_top)
    R *Un, *Vn, *GU, *GV, *Su, *Sv;         // column sums (2-D)
    R *Ub, *Vb, *dE, *paccE, *paccU, *paccV, *gxe, *gye, *corrU, *corrV;
    R *Ub2, *Vb2, *dE2;        // second buffers of the barotropic state (passes ping-pong)
    const R *Hu, *Hv, *rHu, *rHv;
    double *eta, *accE, *accU, *accV;
    // averaging weights a_m of the sub-cycle (null: equal weights 1/N_s) and their first
    // moment sum_m m a_m (the substep is dt / fmom)
    const R* fw;
    double fmom;
    TileMaps tm;               // tensor maps of the state read by the tracer tile
};

// The field pointers of the two tile kernels, passed as one block: a kernel parameter for
// the single model (the code reads them from the parameter bank where used), a copy in
// shared memory for an ensemble item.
template <typename R> struct TracerArgs {
    const R *u, *v, *w, *T, *S;
    R *kap, *GTp, *GSp, *Tn, *Sn;
    const R *dGT, *dGS;
};
template <typename R> struct MomentumArgs {
    const R *u, *v, *w, *pr, *nu, *taux_s, *tauy_s;
    R *Gup, *Gvp, *un, *vn, *cu, *cv, *Un, *Vn, *GU, *GV, *Su, *Sv;
};
template <typename R>
__host__ __device__ inline TracerArgs<R> tracer_args(const StepBuffers<R>& b) {
    return TracerArgs<R>{b.u, b.v, b.w, b.T, b.S, b.kap, b.GT, b.GS, b.Tn, b.Sn, b.dGT, b.dGS};
}
// the v-viscosity's Thomas coefficients go to the scratch field wk, the u-viscosity's to kap
template <typename R>
__host__ __device__ inline MomentumArgs<R> momentum_args(const StepBuffers<R>& b) {
    return MomentumArgs<R>{b.u, b.v, b.w, b.p, b.nu, b.taux_s, b.tauy_s, b.Gu, b.Gv, b.un, b.vn,
                           b.kap, b.wk, b.Un, b.Vn, b.GU, b.GV, b.Su, b.Sv};
}

template <typename R>
void launch_diag(const KP<R>& p, const StepBuffers<R>& b, cudaStream_t s);
template <typename R>
void launch_tracer(const KP<R>& p, const StepBuffers<R>& b, bool step, cudaStream_t s);
template <typename R>
void launch_momentum(const KP<R>& p, const StepBuffers<R>& b, bool step, cudaStream_t s);
template <typename R>
void launch_barotropic(const KP<R>& p, const StepBuffers<R>& b, int ns, double dt, R grav,
                       cudaStream_t s);
template <typename R>
void launch_correct(const KP<R>& p, const StepBuffers<R>& b, cudaStream_t s);
// kernel launches of one barotropic sub-cycle of ns substeps, halos excluded
int baro_passes(int ns);
// averaging weights a_1..a_ns of the sub-cycle for filter `kind` (OCEAN_FILTER_*) into a;
// returns their first moment sum_m m a_m
double baro_filter_weights(int ns, int kind, double* a);
template <typename R>
void launch_halo3(const GeoD& g, R* const* f, int nf, cudaStream_t s);
template <typename R>
void launch_halo2(const GeoD& g, R* f, cudaStream_t s);
// surface wind stress: o[x|y][column] = (R)(t[x|y][j nx + i] * scale) on the padded
// plane (zero where t is null); t is double or float, the product is taken in FP64
template <typename R, typename W>
void launch_wind(const GeoD& g, const W* tx, const W* ty, double scale, R* ox, R* oy,
                 cudaStream_t s);
template <typename R>
int setup_kernel_attributes(int nz);

// FP64 metrics of the conservation reductions (row arrays indexed j + OC_H; per level
// dz, Tref, Sref, dt/dz; per lowest wet level kb = 0..nz the sums from kb to the top of
// Tref dz, Sref dz and dz).
struct DiagMetrics {
    const double *Ac, *dxv, *rdxc, *dz, *Tref, *Sref, *dtdz, *colT, *colS, *colV;
    double dy, rdy, dt;
    // the mixed form's reduction: FP32 copies of the metrics (per level dz, dt/dz; per row
    // Ac, 1/dx_c, dxv, 1/A_c) and the reference part of the totals (sum T dV, sum S dV of
    // the reference profiles, the wet volume), which it adds as constants
    const float *fdz = nullptr, *fdtdz = nullptr, *fAc = nullptr, *frdxc = nullptr,
                *fdxv = nullptr, *frAc = nullptr;
    float fdy = 0.f, frdy = 0.f, fdt = 0.f;
    double cT = 0.0, cS = 0.0, cV = 0.0;
};

// Conservation/health reduction; `partials` is device scratch of at least
// diag_partials_bytes(nx * ny) bytes; `out` (device) receives 8 doubles:
// {sum T dV, sum S dV, sum eta dA, KE, max CFL, nonfinite, wet volume, 0}.
#define OC_DIAG_THREADS 256
size_t diag_partials_bytes(long ncol);   // one partial per block of OC_DIAG_THREADS columns
template <typename R>
void launch_diagnostics(const GeoD& g, const DiagMetrics& m, const R* u, const R* v,
                        const R* T, const R* S, const double* eta, double* partials,
                        double* out, cudaStream_t s);

// Sets the message ocean_last_error(NULL) returns (entry points without a handle).
extern "C" void oc_set_last_error(const char* msg);

// ---- learned closure (ocean_closure.cu, ocean_mlp.cu)
template <typename R>
void launch_closure_features(const KP<R>& p, const R* u, const R* v, const R* T, const R* S,
                             const float* mu, const float* sigma, float* Xf, void* Xb,
                             unsigned char* face, unsigned char* wet, float* dzT, float* dzS,
                             cudaStream_t s);
template <typename R>
void launch_closure_apply(const KP<R>& p, const float* Y, float ks, float gt, float gs, R* kap,
                          R* dGT, R* dGS, cudaStream_t s);
template <typename R>
void launch_coarse_grain(const KP<R>& pf, const KP<R>& pc, int r, const R* uf, const R* vf,
                         const R* Tf, const R* Sf, const R* wf, const R* GTf, const R* GSf,
                         const double* etaf, R* uc, R* vc, R* Tc, R* Sc, double* etac, float* FT,
                         float* FS, float* GTm, float* GSm, cudaStream_t s);
template <typename R>
void launch_closure_targets(const KP<R>& p, const R* GcT, const R* GcS, const float* GTm,
                            const float* GSm, const float* FT, const float* FS, float* GTt,
                            float* GSt, cudaStream_t s);
void closure_forward(const void* Xb, int M, const void* const* Wt, const float* const* b,
                     const int* dims, void* H0, void* H1, float* Y, cudaStream_t s);
void closure_weight_transpose(const float* W, int in, int out, void* Wt, cudaStream_t s);
int closure_gemm_failed();
int tile_wait_failed();
template <typename R> int closure_tiles_setup();
int closure_gemm_setup();

// ---- batched ensemble (kernels in ocean_kernels.cu, host side in ocean_ensemble.cu)
// One member's step parameters and buffers, read by the persistent ensemble kernels from
// a device table (one table per (first step, buffer parity) combination).
template <typename R> struct EnsMember {
    KP<R> k;
    StepBuffers<R> b;
    R dtau;       // barotropic substep 2 dt / (n_substeps + 1)
    double rns;   // 1 / n_substeps
};
// Work item: member m and the position of its unit of work: a column chunk (a), a
// column chunk and level slab (a, b), a tracer/momentum tile (a, b) or a barotropic
// region (a, b).
struct EnsItem { int m, a, b, cost; };
enum {
    ENS_DIAG = 0, ENS_TRACER, ENS_MOMENTUM, ENS_BARO_BEGIN, ENS_BARO_PASS, ENS_BARO_END,
    ENS_CORRECT, ENS_NKIND
};
// Units of work: columns per chunk of the column kernels, tile and region interiors,
// substeps per barotropic pass, levels per slab of the correction.
// chunk: columns of a 2-D item; tile_x, tile_y: a tile item's columns; region_w, region_h:
// a barotropic region including its halo; pass_substeps: the default halo width (= the
// substeps of one pass); corr_slab: levels of a correction item
struct EnsShape { int chunk, tile_x, tile_y, region_w, region_h, pass_substeps, corr_slab; };
// halo widths (substeps per barotropic pass) the ensemble's autotuner chooses among; a
// region's interior is (region_w - 2 bs) x (region_h - 2 bs)
constexpr int ENS_REGION_BS[3] = {4, 6, 8};
EnsShape ens_shape();
// Resident blocks per SM of each ensemble kernel (occupancy calculator).
template <typename R> int ens_blocks_per_sm(int kind);
// One persistent launch of kind `kind` over work[0..nwork): `grid` blocks; items taken in
// order from an atomic counter if `counter` (zeroed beforehand), else blockIdx.x +
// n gridDim.x.  For ENS_BARO_PASS: `odd` selects the ping-pong direction, `nsub` the
// substeps of this pass (at most `bs`, the halo width of the regions the work items were
// cut for).
template <typename R>
void launch_ens(int kind, const EnsMember<R>* mem, const EnsItem* work, int nwork, int grid,
                int* counter, int odd, int nsub, int bs, cudaStream_t s);

// Model internals the ensemble builds on (ocean_api.cu): a model in a caller-provided
// arena on a caller's stream; its sizes and step state; the lowest wet level of column
// (i, j); its table entry for a step from buffer `cur` (first: the Euler start); and
// the bookkeeping after the ensemble has stepped it.
struct OcMemberInfo {
    int nx, ny, nz, px, py, prec, ns, learned, cur;
    long nstep;
    double dt, g;
};
int oc_member_create(const ocean_grid* grid, const double* depth, const ocean_params* params,
                     void* arena, size_t arena_bytes, void* stream, ocean_t* out);
OcMemberInfo oc_member_info(const ocean_s* m);
int oc_member_kb(const ocean_s* m, int i, int j);
template <typename R> EnsMember<R> oc_member_entry(const ocean_s* m, bool first, int cur);
void oc_member_advance(ocean_s* m);
