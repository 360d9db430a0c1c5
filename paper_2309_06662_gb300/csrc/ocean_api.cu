// ocean_api.cu -- host side of libocean's C ABI: validation, metrics and masks, the
// device arena, field transfer and the per-step launch sequence.  All arithmetic of the
// step itself runs in the kernels of ocean_kernels.cu.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ocean.h"
#include "ocean_internal.cuh"

namespace {

thread_local std::string g_last_error;

constexpr double kPi = 3.14159265358979323846;

inline double deg2rad(double d) { return d * (kPi / 180.0); }

struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

struct ocean_s {
    // configuration
    int kind = 0, nx = 0, ny = 0, nz = 0, px = 0, py = 0;
    double x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    std::vector<double> zf, zc, dz;
    ocean_params prm{};
    int prec = OCEAN_FP64;
    size_t esz = 8;
    int pitch = 0;
    long plane = 0, n2pad = 0;
    // device memory
    char* arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device pointers (3-D fields of element size esz)
    void *u[2] = {}, *v[2] = {}, *T[2] = {}, *S[2] = {};
    void *Gu = nullptr, *Gv = nullptr, *GT = nullptr, *GS = nullptr;
    void *w = nullptr, *p = nullptr, *kap = nullptr, *nu = nullptr, *wk = nullptr;
    double* wind_raw = nullptr;   // staging of the host wind stress, [2][ny][nx]
    // 2-D of element size esz
    void *taux_s = nullptr, *tauy_s = nullptr, *Un = nullptr, *Vn = nullptr, *GU = nullptr,
         *GV = nullptr, *Su = nullptr, *Sv = nullptr, *Ub = nullptr, *Vb = nullptr,
         *dE = nullptr, *paccE = nullptr, *paccU = nullptr, *paccV = nullptr, *gxe = nullptr,
         *gye = nullptr, *corrU = nullptr, *corrV = nullptr, *Hu = nullptr, *Hv = nullptr,
         *rHu = nullptr, *rHv = nullptr, *Ub2 = nullptr, *Vb2 = nullptr, *dE2 = nullptr;
    double *eta = nullptr, *accE = nullptr, *accU = nullptr, *accV = nullptr;
    void* fw = nullptr;        // averaging weights of the sub-cycle (power-law filter), R[ns]
    void* vw = nullptr;        // vertical WENO coefficients of each level face, R[(nz+1)*2][OC_VWROW]
    double fmom = 0;           // their first moment sum_m m a_m
    short *kb = nullptr, *kbu = nullptr, *kbv = nullptr, *kbz = nullptr, *kbzin = nullptr;
    void* rowm = nullptr;   // 7 row arrays of (ny + 2H) elements
    void* levm = nullptr;   // 8 level arrays of nz elements
    void* lvt = nullptr;    // per-level rows of OC_LVROW constants of the tile kernels
    double *drow = nullptr, *dlev = nullptr;
    // FP32 metrics of the mixed form's conservation reduction: dz, dt/dz (nz each), Ac
    // (ny + 2H); and the reference part of the totals (sum over wet columns of the
    // reference profiles' content, and the wet volume), formed on the host in FP64
    float* dgf = nullptr;
    double dconst[3] = {0.0, 0.0, 0.0};
    bool dconst_ok = false;
    std::vector<double> h_colT, h_colS, h_colV;
    double *diag_part = nullptr, *diag_out = nullptr;
    // host-side copies
    std::vector<short> h_kb, h_kbu, h_kbv;
    std::vector<double> h_rows[8];   // dxc rdxc dxv rAc rAz fu fv Ac
    std::vector<double> Tref, Sref, h_Hu, h_Hv;
    bool ref_locked = false;   // reference profiles fixed by ocean_set_reference
    // per-phase timing: events recorded on the stream around each phase of a step
    bool prof = false;
    std::vector<std::vector<cudaEvent_t>> prof_pending;
    double phase_ms[OCEAN_NPHASE] = {};
    long prof_steps = 0;
    long launches = 0;         // kernels enqueued by this handle
    // learned closure: network (bf16 W^T per layer, fp32 biases), feature statistics,
    // activations of all columns and the tracer corrections
    int cl_hidden = 0;
    bool cl_ready = false;
    ocean_closure_scales cl_sc{};
    int cl_dims[5] = {};
    void *cl_X = nullptr, *cl_H0 = nullptr, *cl_H1 = nullptr, *cl_Wt[4] = {}, *cl_dGT = nullptr,
         *cl_dGS = nullptr;
    float *cl_Y = nullptr, *cl_b[4] = {}, *cl_stage = nullptr, *cl_mu = nullptr, *cl_sigma = nullptr;   // cl_sigma: 1/sigma
    double dy = 0;
    int cur = 0;
    long nstep = 0;
    bool tend_valid = false;
    // the step as a CUDA graph, per buffer parity and with / without the learned closure
    // (captured on first use; dropped when a launch argument changes)
    cudaGraphExec_t graph[2][2] = {};
    TileMaps tmaps[2];         // tensor maps of the state, per buffer parity
    bool graphs_off = false;   // the stream cannot be captured (the legacy default stream)
    std::string err;
};

namespace {

int fail(ocean_t h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    g_last_error = buf;
    return code;
}

#define OC_CUDA(h, call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, OCEAN_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int validate(const ocean_grid* g, const ocean_params* p) {
    if (!g || !p) return fail(nullptr, OCEAN_ERR_ARG, "null grid or params");
    if (g->kind != 0 && g->kind != 1) return fail(nullptr, OCEAN_ERR_ARG, "grid kind must be 0 or 1");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(nullptr, OCEAN_ERR_ARG, "grid sizes must be >= 1 (got %d x %d x %d)", g->nx, g->ny, g->nz);
    if (g->nz > OC_NZMAX) return fail(nullptr, OCEAN_ERR_ARG, "nz = %d exceeds the maximum %d", g->nz, OC_NZMAX);
    if ((long)g->nx * g->ny > (1L << 30)) return fail(nullptr, OCEAN_ERR_ARG, "too many columns");
    // the tile kernels address a 3-D array (halo and padding included) with 32-bit offsets
    if ((long)((g->nx + 2 * OC_H + 31) & ~31) * (g->ny + 2 * OC_H) * g->nz >= (1L << 31))
        return fail(nullptr, OCEAN_ERR_ARG, "%d x %d x %d cells exceed the 2^31 of a 3-D array",
                    g->nx, g->ny, g->nz);
    if (g->periodic_x && g->nx < OC_H) return fail(nullptr, OCEAN_ERR_ARG, "periodic x needs nx >= %d", OC_H);
    if (g->periodic_y && g->ny < OC_H) return fail(nullptr, OCEAN_ERR_ARG, "periodic y needs ny >= %d", OC_H);
    if (g->periodic_y && g->kind == 1) return fail(nullptr, OCEAN_ERR_ARG, "lat-lon grids cannot be periodic in y");
    if (!(g->x1 > g->x0) || !(g->y1 > g->y0)) return fail(nullptr, OCEAN_ERR_ARG, "empty domain extent");
    if (g->kind == 1 && (g->y0 <= -90.0 || g->y1 >= 90.0))
        return fail(nullptr, OCEAN_ERR_ARG, "latitudes must lie strictly inside (-90, 90)");
    if (!g->z_faces) return fail(nullptr, OCEAN_ERR_ARG, "null z_faces");
    for (int k = 0; k < g->nz; ++k)
        if (!(g->z_faces[k + 1] > g->z_faces[k]))
            return fail(nullptr, OCEAN_ERR_ARG, "z_faces must increase from the bottom to the top");
    if (!(p->dt > 0)) return fail(nullptr, OCEAN_ERR_ARG, "dt must be > 0");
    if (p->n_substeps < 1) return fail(nullptr, OCEAN_ERR_ARG, "n_substeps must be >= 1");
    if (p->precision != OCEAN_FP64 && p->precision != OCEAN_MIXED)
        return fail(nullptr, OCEAN_ERR_ARG, "precision must be OCEAN_FP64 or OCEAN_MIXED");
    if (p->closure != OCEAN_CLOSURE_RI && p->closure != OCEAN_CLOSURE_LEARNED)
        return fail(nullptr, OCEAN_ERR_ARG, "unknown closure");
    if (p->check_every < 0) return fail(nullptr, OCEAN_ERR_ARG, "check_every must be >= 0");
    if (p->closure_hidden < 0 || p->closure_hidden % 16)
        return fail(nullptr, OCEAN_ERR_ARG, "closure_hidden must be 0 or a positive multiple of 16");
    if (p->baro_filter != OCEAN_FILTER_BOXCAR && p->baro_filter != OCEAN_FILTER_POWER_LAW)
        return fail(nullptr, OCEAN_ERR_ARG, "unknown baro_filter %d", p->baro_filter);
    if (p->vertical_weno != OCEAN_VWENO_INDEX && p->vertical_weno != OCEAN_VWENO_STRETCHED)
        return fail(nullptr, OCEAN_ERR_ARG, "unknown vertical_weno %d", p->vertical_weno);
    if (p->momentum_vadv != OCEAN_VADV_CENTRED && p->momentum_vadv != OCEAN_VADV_WENO)
        return fail(nullptr, OCEAN_ERR_ARG, "unknown momentum_vadv %d", p->momentum_vadv);
    return OCEAN_OK;
}

void configure(ocean_t m, const ocean_grid* g, const ocean_params* p) {
    m->kind = g->kind; m->nx = g->nx; m->ny = g->ny; m->nz = g->nz;
    m->px = g->periodic_x ? 1 : 0; m->py = g->periodic_y ? 1 : 0;
    m->x0 = g->x0; m->x1 = g->x1; m->y0 = g->y0; m->y1 = g->y1;
    m->zf.assign(g->z_faces, g->z_faces + g->nz + 1);
    m->zc.resize(g->nz); m->dz.resize(g->nz);
    for (int k = 0; k < g->nz; ++k) {
        m->zc[k] = 0.5 * (m->zf[k] + m->zf[k + 1]);
        m->dz[k] = m->zf[k + 1] - m->zf[k];
    }
    m->prm = *p;
    m->prm.taux = nullptr;
    m->prm.tauy = nullptr;
    m->prec = p->precision;
    m->esz = p->precision == OCEAN_FP64 ? sizeof(double) : sizeof(float);
    int w = g->nx + 2 * OC_H;
    m->pitch = (w + 31) & ~31;
    m->n2pad = (long)m->pitch * (g->ny + 2 * OC_H);
    m->plane = m->n2pad;
    m->Tref.assign(g->nz, p->T0);
    m->Sref.assign(g->nz, p->S0);
}

// lays out (base == nullptr: sizes) every device array; returns the total bytes
size_t layout(ocean_t m, char* base) {
    Carver c{base};
    const size_t n3 = (size_t)m->plane * m->nz, n2 = (size_t)m->n2pad, e = m->esz;
    auto f3 = [&]() { return (void*)c.take<char>(n3 * e); };
    auto f2 = [&]() { return (void*)c.take<char>(n2 * e); };
    for (int b = 0; b < 2; ++b) { m->u[b] = f3(); m->v[b] = f3(); m->T[b] = f3(); m->S[b] = f3(); }
    m->Gu = f3(); m->Gv = f3(); m->GT = f3(); m->GS = f3();
    m->w = f3(); m->p = f3(); m->kap = f3(); m->nu = f3(); m->wk = f3();
    m->wind_raw = c.take<double>(2 * (size_t)m->nx * m->ny);
    void** two[] = {&m->taux_s, &m->tauy_s, &m->Un, &m->Vn, &m->GU, &m->GV, &m->Su, &m->Sv,
                    &m->Ub, &m->Vb, &m->dE, &m->paccE, &m->paccU, &m->paccV, &m->gxe, &m->gye,
                    &m->corrU, &m->corrV, &m->Hu, &m->Hv, &m->rHu, &m->rHv, &m->Ub2, &m->Vb2,
                    &m->dE2};
    for (void** q : two) *q = f2();
    m->fw = c.take<char>((size_t)m->prm.n_substeps * e);
    m->vw = c.take<char>(((size_t)m->nz + 1) * 2 * OC_VWROW * e);
    m->eta = c.take<double>(n2); m->accE = c.take<double>(n2);
    m->accU = c.take<double>(n2); m->accV = c.take<double>(n2);
    m->kb = c.take<short>(n2); m->kbu = c.take<short>(n2); m->kbv = c.take<short>(n2);
    m->kbz = c.take<short>(n2); m->kbzin = c.take<short>(n2);
    const size_t nr = (size_t)m->ny + 2 * OC_H;
    m->rowm = c.take<char>(7 * nr * e);
    m->levm = c.take<char>(8 * (size_t)m->nz * e);
    m->lvt = c.take<char>((size_t)OC_LVROW * m->nz * e);
    m->drow = c.take<double>(3 * nr);
    m->dlev = c.take<double>(4 * (size_t)m->nz + 3 * ((size_t)m->nz + 1));
    m->dgf = c.take<float>(2 * (size_t)m->nz + nr);
    m->diag_part = reinterpret_cast<double*>(c.take<char>(diag_partials_bytes((long)m->nx * m->ny)));
    m->diag_out = c.take<double>(8);
    m->cl_mu = c.take<float>(6 * (size_t)m->nz);
    m->cl_sigma = c.take<float>(6 * (size_t)m->nz);
    m->cl_hidden = m->prm.closure_hidden;
    if (m->cl_hidden > 0) {
        const int H = m->cl_hidden, nz = m->nz;
        const int d[5] = {6 * nz, H, H, H, 3 * nz};
        for (int q = 0; q < 5; ++q) m->cl_dims[q] = d[q];
        const size_t M = (size_t)m->nx * m->ny;
        m->cl_X = c.take<char>(M * d[0] * 2);
        m->cl_H0 = c.take<char>(M * H * 2);
        m->cl_H1 = c.take<char>(M * H * 2);
        m->cl_Y = c.take<float>(M * d[4]);
        size_t big = 0;
        for (int l = 0; l < 4; ++l) {
            m->cl_Wt[l] = c.take<char>((size_t)d[l] * d[l + 1] * 2);
            m->cl_b[l] = c.take<float>(d[l + 1]);
            big = std::max(big, (size_t)d[l] * d[l + 1]);
        }
        m->cl_stage = c.take<float>(big);
        m->cl_dGT = f3();
        m->cl_dGS = f3();
    }
    return c.off + 256;
}

inline long hix2(const ocean_t m, int i, int j) {
    return (long)(j + OC_H) * m->pitch + (i + OC_H);
}

// wrap a padded column index onto the interior; false when it lies beyond a wall
inline bool wrap(const ocean_t m, int& i, int& j) {
    if (m->px) { i %= m->nx; if (i < 0) i += m->nx; }
    else if (i < 0 || i >= m->nx) return false;
    if (m->py) { j %= m->ny; if (j < 0) j += m->ny; }
    else if (j < 0 || j >= m->ny) return false;
    return true;
}

// host -> device copy on the handle's stream, complete on return
void upload_bytes(ocean_t m, void* dst, const void* src, size_t bytes) {
    cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, m->stream);
    cudaStreamSynchronize(m->stream);
}

template <typename R>
void upload_conv(ocean_t m, const std::vector<double>& src, void* dst) {
    std::vector<R> t(src.size());
    for (size_t q = 0; q < src.size(); ++q) t[q] = (R)src[q];
    upload_bytes(m, dst, t.data(), t.size() * sizeof(R));
}

void upload_real(ocean_t m, const std::vector<double>& src, void* dst) {
    if (m->prec == OCEAN_FP64) upload_conv<double>(m, src, dst);
    else upload_conv<float>(m, src, dst);
}

// Weights c[0..n-1] for which sum_j c_j qbar_j is the value at xf of the polynomial of
// degree n-1 with means qbar_j over the n cells between the edges e[0..n] (monotone in
// either direction): with the primitive P(x) = int_{e_0}^x p, known at the edges as
// P(e_m) = sum_{j<m} (e_{j+1} - e_j) qbar_j, interpolate P by the Lagrange polynomial
// through the n+1 edges and differentiate: p(xf) = sum_m P(e_m) L_m'(xf), so
// c_j = (e_{j+1} - e_j) sum_{m>j} L_m'(xf).  Coordinates are shifted to xf and scaled by
// the mean cell width first (the weights do not depend on either).
void face_weights(int n, const double* e, double xf, double* c) {
    double s[6], dL[6];
    const double h = std::fabs(e[n] - e[0]) / n;
    for (int m = 0; m <= n; ++m) s[m] = (e[m] - xf) / h;
    for (int m = 0; m <= n; ++m) {
        double den = 1.0, num = 0.0;
        for (int l = 0; l <= n; ++l) {
            if (l == m) continue;
            den *= s[m] - s[l];
            double pr = 1.0;   // prod over q != m, l of (0 - s_q)
            for (int q = 0; q <= n; ++q)
                if (q != m && q != l) pr *= -s[q];
            num += pr;
        }
        dL[m] = num / den / h;
    }
    for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int m = j + 1; m <= n; ++m) acc += dL[m];
        c[j] = (e[j + 1] - e[j]) * acc;
    }
}

// One row of the vertical WENO table: the reconstruction at level face kf upwind by
// direction dir (0: the face velocity is >= 0 and the stencil lies below, cells kf-3 ..
// kf+1; 1: above, cells kf+2 .. kf-2), ordered from upwind to downwind.  The fifth-order
// part is filled when all six edges exist, the third-order part when its four do; the
// kernels use a part only where its stencil lies in the fluid, so inside the grid.
void vw_row(const std::vector<double>& zf, int kf, int dir, double* row) {
    const int nz = (int)zf.size() - 1;
    for (int n = 0; n < OC_VWROW; ++n) row[n] = 0.0;
    double e[6];
    bool have[6];
    for (int n = 0; n < 6; ++n) {
        const int ke = dir == 0 ? kf - 3 + n : kf + 3 - n;
        have[n] = ke >= 0 && ke <= nz;
        e[n] = have[n] ? zf[ke] : 0.0;
    }
    const double xf = zf[kf];
    if (have[0] && have[5]) {
        double c5[5];
        for (int r = 0; r < 3; ++r) face_weights(3, e + r, xf, row + 3 * r);
        face_weights(5, e, xf, c5);
        row[9] = c5[0] / row[0];
        row[11] = c5[4] / row[8];
        row[10] = 1.0 - row[9] - row[11];
    }
    if (have[1] && have[4]) {
        double c3[3];
        face_weights(2, e + 1, xf, row + 12);
        face_weights(2, e + 2, xf, row + 14);
        face_weights(3, e + 1, xf, c3);
        row[16] = c3[0] / row[12];
        row[17] = 1.0 - row[16];
    }
}

void upload_levels(ocean_t m) {
    const int nz = m->nz;
    std::vector<double> lv(8 * (size_t)nz, 0.0), dl(4 * (size_t)nz + 3 * ((size_t)nz + 1), 0.0);
    for (int k = 0; k < nz; ++k) {
        lv[k] = m->dz[k];
        lv[nz + k] = 1.0 / m->dz[k];
        lv[2 * nz + k] = k > 0 ? m->zc[k] - m->zc[k - 1] : 0.0;
        lv[3 * nz + k] = k > 0 ? 1.0 / (m->zc[k] - m->zc[k - 1]) : 0.0;
        lv[4 * nz + k] = m->Tref[k];
        lv[5 * nz + k] = m->Sref[k];
        lv[6 * nz + k] = k > 0 ? m->Tref[k] - m->Tref[k - 1] : 0.0;
        lv[7 * nz + k] = k > 0 ? m->Sref[k] - m->Sref[k - 1] : 0.0;
        dl[k] = m->dz[k];
        dl[nz + k] = m->Tref[k];
        dl[2 * nz + k] = m->Sref[k];
        dl[3 * nz + k] = m->prm.dt / m->dz[k];
    }
    // sums from level kb to the top, kb = 0 .. nz: of Tref dz, Sref dz and dz (the
    // reference part of a column's tracer content and its volume per unit area)
    double* cT = dl.data() + 4 * nz;
    double* cS = cT + nz + 1;
    double* cV = cS + nz + 1;
    for (int k = nz - 1; k >= 0; --k) {
        cT[k] = cT[k + 1] + m->Tref[k] * m->dz[k];
        cS[k] = cS[k + 1] + m->Sref[k] * m->dz[k];
        cV[k] = cV[k + 1] + m->dz[k];
    }
    upload_real(m, lv, m->levm);
    upload_bytes(m, m->dlev, dl.data(), dl.size() * sizeof(double));
    std::vector<float> fl(2 * (size_t)nz);
    for (int k = 0; k < nz; ++k) {
        fl[k] = (float)m->dz[k];
        fl[nz + k] = (float)(m->prm.dt / m->dz[k]);
    }
    upload_bytes(m, m->dgf, fl.data(), fl.size() * sizeof(float));
    m->h_colT.assign(cT, cT + nz + 1);
    m->h_colS.assign(cS, cS + nz + 1);
    m->h_colV.assign(cV, cV + nz + 1);
    m->dconst_ok = false;
    // rows of the tile kernels (KP::lvt): dz, 1/dz, dt/(dz dzf) below and above, Tref,
    // Sref, and those factors times the reference profiles' level differences
    std::vector<double> rows((size_t)OC_LVROW * nz, 0.0);
    for (int k = 0; k < nz; ++k) {
        double* r = rows.data() + (size_t)k * OC_LVROW;
        const double alo = k > 0 ? m->prm.dt / (m->dz[k] * (m->zc[k] - m->zc[k - 1])) : 0.0;
        const double ahi = k < nz - 1 ? m->prm.dt / (m->dz[k] * (m->zc[k + 1] - m->zc[k])) : 0.0;
        r[0] = m->dz[k];
        r[1] = 1.0 / m->dz[k];
        r[2] = alo;
        r[3] = ahi;
        r[4] = m->Tref[k];
        r[5] = m->Sref[k];
        r[6] = k < nz - 1 ? ahi * (m->Tref[k + 1] - m->Tref[k]) : 0.0;
        r[7] = k > 0 ? alo * (m->Tref[k] - m->Tref[k - 1]) : 0.0;
        r[8] = k < nz - 1 ? ahi * (m->Sref[k + 1] - m->Sref[k]) : 0.0;
        r[9] = k > 0 ? alo * (m->Sref[k] - m->Sref[k - 1]) : 0.0;
    }
    upload_real(m, rows, m->lvt);
    std::vector<double> vw(((size_t)nz + 1) * 2 * OC_VWROW);
    for (int kf = 0; kf <= nz; ++kf)
        for (int dir = 0; dir < 2; ++dir) vw_row(m->zf, kf, dir, vw.data() + ((size_t)kf * 2 + dir) * OC_VWROW);
    upload_real(m, vw, m->vw);
}

// metrics, masks, column depths; host FP64, uploaded once
int build_geometry(ocean_t m, const double* depth) {
    const int nx = m->nx, ny = m->ny, nz = m->nz, H = OC_H;
    const int nr = ny + 2 * H;
    const ocean_params& p = m->prm;
    // ---- rows
    for (auto& r : m->h_rows) r.assign(nr, 0.0);
    double dy;
    if (m->kind == 0) {
        const double dx = (m->x1 - m->x0) / nx;
        dy = (m->y1 - m->y0) / ny;
        const double ymid = 0.5 * (m->y0 + m->y1);
        for (int jj = 0; jj < nr; ++jj) {
            const int j = jj - H;
            m->h_rows[0][jj] = dx;
            m->h_rows[2][jj] = dx;
            m->h_rows[5][jj] = p.f0 + p.beta_plane * (m->y0 + (j + 0.5) * dy - ymid);
            m->h_rows[6][jj] = p.f0 + p.beta_plane * (m->y0 + j * dy - ymid);
        }
    } else {
        const double dlam = deg2rad((m->x1 - m->x0) / nx), dphi = (m->y1 - m->y0) / ny;
        dy = p.radius * deg2rad(dphi);
        for (int jj = 0; jj < nr; ++jj) {
            const int j = jj - H;
            const double pc = deg2rad(m->y0 + (j + 0.5) * dphi), pf = deg2rad(m->y0 + j * dphi);
            m->h_rows[0][jj] = p.radius * std::fmax(std::cos(pc), 1e-12) * dlam;
            m->h_rows[2][jj] = p.radius * std::fmax(std::cos(pf), 1e-12) * dlam;
            m->h_rows[5][jj] = 2.0 * p.omega * std::sin(pc);
            m->h_rows[6][jj] = 2.0 * p.omega * std::sin(pf);
        }
    }
    m->dy = dy;
    for (int jj = 0; jj < nr; ++jj) {
        m->h_rows[1][jj] = 1.0 / m->h_rows[0][jj];
        m->h_rows[7][jj] = m->h_rows[0][jj] * dy;
        m->h_rows[3][jj] = 1.0 / m->h_rows[7][jj];
        m->h_rows[4][jj] = 1.0 / (m->h_rows[2][jj] * dy);
    }
    std::vector<double> rows(7 * (size_t)nr);
    for (int a = 0; a < 7; ++a)
        for (int jj = 0; jj < nr; ++jj) rows[(size_t)a * nr + jj] = m->h_rows[a][jj];
    upload_real(m, rows, m->rowm);
    std::vector<double> drow(3 * (size_t)nr);
    for (int jj = 0; jj < nr; ++jj) {
        drow[jj] = m->h_rows[7][jj];
        drow[nr + jj] = m->h_rows[2][jj];
        drow[2 * nr + jj] = m->h_rows[1][jj];
    }
    upload_bytes(m, m->drow, drow.data(), drow.size() * sizeof(double));
    std::vector<float> acf((size_t)nr);
    for (int jj = 0; jj < nr; ++jj) acf[jj] = (float)m->h_rows[7][jj];
    upload_bytes(m, m->dgf + 2 * (size_t)m->nz, acf.data(), acf.size() * sizeof(float));
    upload_levels(m);
    // ---- averaging weights of the sub-cycle
    std::vector<double> fw((size_t)p.n_substeps);
    m->fmom = baro_filter_weights(p.n_substeps, p.baro_filter, fw.data());
    upload_real(m, fw, m->fw);
    // ---- masks
    const long n2 = m->n2pad;
    std::vector<short> kbi((size_t)nx * ny);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double d = depth[(size_t)j * nx + i];
            if (!(d >= 0.0) || !std::isfinite(d))
                return fail(nullptr, OCEAN_ERR_ARG, "depth must be finite and >= 0 (column %d,%d)", i, j);
            int kb = nz;
            if (d >= p.min_depth)
                for (int k = nz - 1; k >= 0 && m->zc[k] > -d; --k) kb = k;
            kbi[(size_t)j * nx + i] = (short)kb;
        }
    auto KB = [&](int i, int j) -> int {
        if (!wrap(m, i, j)) return nz;
        return kbi[(size_t)j * nx + i];
    };
    m->h_kb.assign(n2, (short)nz);
    m->h_kbu.assign(n2, (short)nz);
    m->h_kbv.assign(n2, (short)nz);
    std::vector<short> kbz(n2, (short)nz), kbzin(n2, (short)nz);
    for (int j = -H; j < ny + H; ++j)
        for (int i = -H; i < nx + H; ++i) {
            const long c = hix2(m, i, j);
            const int a = KB(i, j), b = KB(i - 1, j), cc = KB(i, j - 1), d = KB(i - 1, j - 1);
            m->h_kb[c] = (short)a;
            m->h_kbu[c] = (short)std::max(a, b);
            m->h_kbv[c] = (short)std::max(a, cc);
            kbz[c] = (short)std::max(std::max(a, b), std::max(cc, d));
            kbzin[c] = (short)std::min(std::min(a, b), std::min(cc, d));
        }
    upload_bytes(m, m->kb, m->h_kb.data(), n2 * sizeof(short));
    upload_bytes(m, m->kbu, m->h_kbu.data(), n2 * sizeof(short));
    upload_bytes(m, m->kbv, m->h_kbv.data(), n2 * sizeof(short));
    upload_bytes(m, m->kbz, kbz.data(), n2 * sizeof(short));
    upload_bytes(m, m->kbzin, kbzin.data(), n2 * sizeof(short));
    // ---- column depths
    m->h_Hu.assign(n2, 0.0);
    m->h_Hv.assign(n2, 0.0);
    std::vector<double> rHu(n2, 0.0), rHv(n2, 0.0);
    for (long c = 0; c < n2; ++c) {
        double hu = 0, hv = 0;
        for (int k = m->h_kbu[c]; k < nz; ++k) hu += m->dz[k];
        for (int k = m->h_kbv[c]; k < nz; ++k) hv += m->dz[k];
        m->h_Hu[c] = hu; m->h_Hv[c] = hv;
        rHu[c] = hu > 0 ? 1.0 / hu : 0.0;
        rHv[c] = hv > 0 ? 1.0 / hv : 0.0;
    }
    upload_real(m, m->h_Hu, m->Hu);
    upload_real(m, m->h_Hv, m->Hv);
    upload_real(m, rHu, m->rHu);
    upload_real(m, rHv, m->rHv);
    return OCEAN_OK;
}

// The host arrays go to a device staging area by two copies on the model's stream; a
// kernel scales them by 1 / (rho0 dz_top) and writes them into the padded fields.
// Returns once the host arrays have been read.  W: double, or float (half the bytes).
template <typename W>
int set_wind(ocean_t m, const W* taux, const W* tauy) {
    const size_t n = (size_t)m->nx * m->ny;
    W* raw = reinterpret_cast<W*>(m->wind_raw);   // room for 2 n doubles
    if (taux)
        OC_CUDA(m, cudaMemcpyAsync(raw, taux, n * sizeof(W), cudaMemcpyHostToDevice, m->stream));
    if (tauy)
        OC_CUDA(m, cudaMemcpyAsync(raw + n, tauy, n * sizeof(W), cudaMemcpyHostToDevice, m->stream));
    const double s = 1.0 / (m->prm.rho0 * m->dz[m->nz - 1]);
    GeoD g{};
    g.nx = m->nx; g.ny = m->ny; g.nz = m->nz; g.px = m->px; g.py = m->py; g.pitch = m->pitch;
    g.plane = m->plane;
    if (m->prec == OCEAN_FP64)
        launch_wind<double, W>(g, taux ? raw : nullptr, tauy ? raw + n : nullptr, s,
                               reinterpret_cast<double*>(m->taux_s),
                               reinterpret_cast<double*>(m->tauy_s), m->stream);
    else
        launch_wind<float, W>(g, taux ? raw : nullptr, tauy ? raw + n : nullptr, s,
                              reinterpret_cast<float*>(m->taux_s),
                              reinterpret_cast<float*>(m->tauy_s), m->stream);
    OC_CUDA(m, cudaGetLastError());
    OC_CUDA(m, cudaStreamSynchronize(m->stream));
    return OCEAN_OK;
}

// field location and mask: which lowest-wet-level array applies (0 cell, 1 u, 2 v)
struct FieldRef {
    void* ptr = nullptr;
    bool is2d = false, is_double = false, readonly = false;
    int mask = 0;
};

FieldRef field_ref(ocean_t m, int id) {
    FieldRef r;
    const int c = m->cur, n = 1 - m->cur;
    switch (id) {
        case OCEAN_U: r.ptr = m->u[c]; r.mask = 1; break;
        case OCEAN_V: r.ptr = m->v[c]; r.mask = 2; break;
        case OCEAN_T: r.ptr = m->T[c]; break;
        case OCEAN_S: r.ptr = m->S[c]; break;
        case OCEAN_ETA: r.ptr = m->eta; r.is2d = true; r.is_double = true; break;
        case OCEAN_GU_PREV: r.ptr = m->Gu; r.mask = 1; break;
        case OCEAN_GV_PREV: r.ptr = m->Gv; r.mask = 2; break;
        case OCEAN_GT_PREV: r.ptr = m->GT; break;
        case OCEAN_GS_PREV: r.ptr = m->GS; break;
        case OCEAN_W: r.ptr = m->w; r.readonly = true; break;
        case OCEAN_P: r.ptr = m->p; r.readonly = true; break;
        case OCEAN_KAPPA: r.ptr = m->kap; r.readonly = true; break;
        case OCEAN_NU: r.ptr = m->nu; r.readonly = true; break;
        case OCEAN_GU: r.ptr = m->u[n]; r.mask = 1; r.readonly = true; break;
        case OCEAN_GV: r.ptr = m->v[n]; r.mask = 2; r.readonly = true; break;
        case OCEAN_GT: r.ptr = m->T[n]; r.readonly = true; break;
        case OCEAN_GS: r.ptr = m->S[n]; r.readonly = true; break;
        case OCEAN_HU: r.ptr = m->Hu; r.is2d = true; r.readonly = true; break;
        case OCEAN_HV: r.ptr = m->Hv; r.is2d = true; r.readonly = true; break;
        case OCEAN_T_ANOM: r.ptr = m->T[c]; break;
        case OCEAN_S_ANOM: r.ptr = m->S[c]; break;
        default: break;
    }
    return r;
}

// kinematic pressure of the reference profiles, added back on output
std::vector<double> reference_pressure(const ocean_t m) {
    const int nz = m->nz;
    const ocean_params& p = m->prm;
    std::vector<double> P(nz), b(nz);
    for (int k = 0; k < nz; ++k)
        b[k] = p.g * (p.alpha * (m->Tref[k] - p.T0) - p.beta_s * (m->Sref[k] - p.S0));
    P[nz - 1] = -b[nz - 1] * (m->zf[nz] - m->zc[nz - 1]);
    for (int k = nz - 2; k >= 0; --k) P[k] = P[k + 1] - 0.5 * (b[k] + b[k + 1]) * (m->zc[k + 1] - m->zc[k]);
    return P;
}

template <typename R>
KP<R> make_kp(const ocean_t m, bool first) {
    KP<R> k{};
    GeoD& g = k.g;
    g.nx = m->nx; g.ny = m->ny; g.nz = m->nz; g.px = m->px; g.py = m->py; g.pitch = m->pitch;
    g.plane = m->plane;
    g.kb = m->kb; g.kbu = m->kbu; g.kbv = m->kbv; g.kbz = m->kbz; g.kbzin = m->kbzin;
    const size_t nr = (size_t)m->ny + 2 * OC_H;
    const R* rows = reinterpret_cast<const R*>(m->rowm);
    k.dxc = rows; k.rdxc = rows + nr; k.dxv = rows + 2 * nr; k.rAc = rows + 3 * nr;
    k.rAz = rows + 4 * nr; k.fu = rows + 5 * nr; k.fv = rows + 6 * nr;
    const R* lv = reinterpret_cast<const R*>(m->levm);
    const int nz = m->nz;
    k.dz = lv; k.rdz = lv + nz; k.dzf = lv + 2 * nz; k.rdzf = lv + 3 * nz;
    k.Tref = lv + 4 * nz; k.Sref = lv + 5 * nz; k.dTref = lv + 6 * nz; k.dSref = lv + 7 * nz;
    const ocean_params& p = m->prm;
    k.dy = (R)m->dy; k.rdy = (R)(1.0 / m->dy); k.dt = (R)p.dt;
    k.ca = first ? R(1) : (R)(1.5 + p.chi);
    k.cb = first ? R(0) : (R)(0.5 + p.chi);
    k.grav = (R)p.g; k.alpha = (R)p.alpha; k.beta_s = (R)p.beta_s;
    k.nu0 = (R)p.nu0; k.ri_a = (R)p.ri_a; k.nu_b = (R)p.nu_b; k.kappa_b = (R)p.kappa_b;
    k.kappa_conv = (R)p.kappa_conv; k.eps = (R)p.weno_eps;
    k.ptop = (R)(m->zf[nz] - m->zc[nz - 1]);
    k.linear = p.weno_linear;
    k.vw = reinterpret_cast<const R*>(m->vw);
    k.vweno = p.vertical_weno;
    k.mvadv = p.momentum_vadv;
    k.lvt = reinterpret_cast<const R*>(m->lvt);
    return k;
}

// buffers of a step from state buffer `cur` (default: the current one)
template <typename R>
StepBuffers<R> make_bufs(const ocean_t m, int cur = -1) {
    StepBuffers<R> b{};
    const int c = cur < 0 ? m->cur : cur, n = 1 - c;
    auto P = [](void* q) { return reinterpret_cast<R*>(q); };
    b.u = P(m->u[c]); b.v = P(m->v[c]); b.T = P(m->T[c]); b.S = P(m->S[c]);
    b.un = P(m->u[n]); b.vn = P(m->v[n]); b.Tn = P(m->T[n]); b.Sn = P(m->S[n]);
    b.Gu = P(m->Gu); b.Gv = P(m->Gv); b.GT = P(m->GT); b.GS = P(m->GS);
    b.w = P(m->w); b.p = P(m->p); b.kap = P(m->kap); b.nu = P(m->nu); b.wk = P(m->wk);
    b.taux_s = P(m->taux_s); b.tauy_s = P(m->tauy_s);
    b.Un = P(m->Un); b.Vn = P(m->Vn); b.GU = P(m->GU); b.GV = P(m->GV); b.Su = P(m->Su); b.Sv = P(m->Sv);
    b.Ub = P(m->Ub); b.Vb = P(m->Vb); b.dE = P(m->dE); b.paccE = P(m->paccE);
    b.paccU = P(m->paccU); b.paccV = P(m->paccV); b.gxe = P(m->gxe); b.gye = P(m->gye);
    b.corrU = P(m->corrU); b.corrV = P(m->corrV);
    b.Ub2 = P(m->Ub2); b.Vb2 = P(m->Vb2); b.dE2 = P(m->dE2);
    b.Hu = P(m->Hu); b.Hv = P(m->Hv); b.rHu = P(m->rHu); b.rHv = P(m->rHv);
    b.eta = m->eta; b.accE = m->accE; b.accU = m->accU; b.accV = m->accV;
    b.fw = m->prm.baro_filter == OCEAN_FILTER_BOXCAR ? nullptr : reinterpret_cast<const R*>(m->fw);
    b.fmom = m->fmom;
    b.tm = m->tmaps[c];
    return b;
}

// tensor maps of T, S, u, v of both buffer parities (3-D views of the padded fields)
bool build_tile_maps(ocean_t m) {
    const CUtensorMapDataType dt =
        m->prec == OCEAN_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const unsigned long long dims[3] = {(unsigned long long)m->pitch,
                                        (unsigned long long)(m->ny + 2 * OC_H),
                                        (unsigned long long)m->nz};
    const unsigned long long strides[2] = {(unsigned long long)m->pitch * m->esz,
                                           (unsigned long long)m->plane * m->esz};
    // boxes of one level: the tracer's T, S with a 3-cell halo read from i0 - 4 (a 16-byte
    // aligned start), its u- and v-face velocities; the momentum's u (rows j0-3 ..), v
    // (rows j0-2 ..), the centred p, w, nu (rows j0-1 ..); the block's own columns
    const unsigned TXu = OC_TX, TYu = OC_TY;
    const unsigned boxTS[3] = {TXu + 8, TYu + 6, 1}, boxU[3] = {TXu + 4, TYu, 1},
                   boxV[3] = {TXu, TYu + 1, 1}, boxMU[3] = {TXu + 8, TYu + 6, 1},
                   boxMV[3] = {TXu + 8, TYu + 5, 1}, boxC[3] = {TXu + 4, TYu + 1, 1},
                   boxO[3] = {TXu, TYu, 1};
    const CUtensorMapSwizzle no = CU_TENSOR_MAP_SWIZZLE_NONE;
    for (int c = 0; c < 2; ++c) {
        TileMaps& t = m->tmaps[c];
        if (!oc_encode_tiled(&t.T, dt, 3, m->T[c], dims, strides, boxTS, no) ||
            !oc_encode_tiled(&t.S, dt, 3, m->S[c], dims, strides, boxTS, no) ||
            !oc_encode_tiled(&t.tu, dt, 3, m->u[c], dims, strides, boxU, no) ||
            !oc_encode_tiled(&t.tv, dt, 3, m->v[c], dims, strides, boxV, no) ||
            !oc_encode_tiled(&t.tw, dt, 3, m->w, dims, strides, boxO, no) ||
            !oc_encode_tiled(&t.tk, dt, 3, m->kap, dims, strides, boxO, no) ||
            !oc_encode_tiled(&t.tgt, dt, 3, m->GT, dims, strides, boxO, no) ||
            !oc_encode_tiled(&t.tgs, dt, 3, m->GS, dims, strides, boxO, no) ||
            !oc_encode_tiled(&t.mu, dt, 3, m->u[c], dims, strides, boxMU, no) ||
            !oc_encode_tiled(&t.mv, dt, 3, m->v[c], dims, strides, boxMV, no) ||
            !oc_encode_tiled(&t.mp, dt, 3, m->p, dims, strides, boxC, no) ||
            !oc_encode_tiled(&t.mw, dt, 3, m->w, dims, strides, boxC, no) ||
            !oc_encode_tiled(&t.mnu, dt, 3, m->nu, dims, strides, boxC, no) ||
            !oc_encode_tiled(&t.mgu, dt, 3, m->Gu, dims, strides, boxO, no) ||
            !oc_encode_tiled(&t.mgv, dt, 3, m->Gv, dims, strides, boxO, no))
            return false;
    }
    return true;
}

// kernels one step enqueues (each periodic direction adds one halo kernel per halo fill)
long launches_per_step(const ocean_t m) {
    const long hk = (m->px ? 1 : 0) + (m->py ? 1 : 0);
    const long ns = m->prm.n_substeps;
    return 3 + (hk + 1 + baro_passes((int)ns) + 1) + 1 + hk;
}

// the learned closure after the Richardson-number closure: network on every column, then
// its diffusivity added to kap and its tracer corrections into b.dGT, b.dGS
template <typename R>
bool enqueue_closure(ocean_t m, const KP<R>& k, StepBuffers<R>& b) {
    if (!(m->cl_ready && m->prm.closure == OCEAN_CLOSURE_LEARNED)) return false;
    cudaStream_t s = m->stream;
    launch_closure_features<R>(k, b.u, b.v, b.T, b.S, m->cl_mu, m->cl_sigma, nullptr, m->cl_X,
                               nullptr, nullptr, nullptr, nullptr, s);
    closure_forward(m->cl_X, m->nx * m->ny, m->cl_Wt, m->cl_b, m->cl_dims, m->cl_H0, m->cl_H1,
                    m->cl_Y, s);
    launch_closure_apply<R>(k, m->cl_Y, m->cl_sc.kappa, m->cl_sc.gT, m->cl_sc.gS, b.kap,
                            reinterpret_cast<R*>(m->cl_dGT), reinterpret_cast<R*>(m->cl_dGS), s);
    b.dGT = reinterpret_cast<const R*>(m->cl_dGT);
    b.dGS = reinterpret_cast<const R*>(m->cl_dGS);
    return true;
}

bool closure_on(const ocean_t m) { return m->cl_ready && m->prm.closure == OCEAN_CLOSURE_LEARNED; }

// kernels one step enqueues, the learned closure's six included
long step_launches(const ocean_t m) { return launches_per_step(m) + (closure_on(m) ? 6 : 0); }

void drop_graphs(ocean_t m) {
    for (auto& row : m->graph)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

// the kernels of one step from buffer m->cur (with profiling events when `ev`)
template <typename R>
void launch_step(ocean_t m, bool first, std::vector<cudaEvent_t>* ev) {
    const KP<R> k = make_kp<R>(m, first);
    StepBuffers<R> b = make_bufs<R>(m);
    cudaStream_t s = m->stream;
    auto mark = [&]() {
        if (!ev) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev->push_back(e);
    };
    mark();
    launch_diag<R>(k, b, s);
    enqueue_closure<R>(m, k, b);
    mark();
    launch_tracer<R>(k, b, true, s);
    mark();
    launch_momentum<R>(k, b, true, s);
    mark();
    launch_barotropic<R>(k, b, m->prm.n_substeps, m->prm.dt, (R)m->prm.g, s);
    mark();
    launch_correct<R>(k, b, s);
    if (m->px || m->py) {
        R* f[4] = {b.un, b.vn, b.Tn, b.Sn};
        launch_halo3<R>(k.g, f, 4, s);
    }
    mark();
}

// One step: direct launches for the first (Euler) step and while profiling, else the
// step's CUDA graph for this buffer parity (captured on first use).
template <typename R>
int enqueue_step(ocean_t m) {
    const bool first = m->nstep == 0;
    if (first || m->prof || m->graphs_off) {
        std::vector<cudaEvent_t> ev;
        launch_step<R>(m, first, m->prof ? &ev : nullptr);
        if (m->prof) m->prof_pending.push_back(ev);
    } else {
        cudaGraphExec_t& g = m->graph[m->cur][closure_on(m) ? 1 : 0];
        if (!g) {
            cudaGraph_t gr = nullptr;
            if (cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                (void)cudaGetLastError();   // not capturable: launch directly from now on
                m->graphs_off = true;
                launch_step<R>(m, false, nullptr);
            } else {
                launch_step<R>(m, false, nullptr);
                cudaError_t e = cudaStreamEndCapture(m->stream, &gr);
                if (e == cudaSuccess) e = cudaGraphInstantiate(&g, gr, 0);
                if (gr) cudaGraphDestroy(gr);
                if (e != cudaSuccess) {
                    g = nullptr;
                    return fail(m, OCEAN_ERR_CUDA, "step graph capture failed: %s", cudaGetErrorString(e));
                }
            }
        }
        if (g) {
            cudaError_t e = cudaGraphLaunch(g, m->stream);
            if (e != cudaSuccess)
                return fail(m, OCEAN_ERR_CUDA, "cudaGraphLaunch failed: %s", cudaGetErrorString(e));
        }
    }
    m->launches += step_launches(m);
    m->cur = 1 - m->cur;
    m->nstep += 1;
    m->tend_valid = false;
    return OCEAN_OK;
}

template <typename R>
void enqueue_tendencies(ocean_t m) {
    const KP<R> k = make_kp<R>(m, m->nstep == 0);
    StepBuffers<R> b = make_bufs<R>(m);
    launch_diag<R>(k, b, m->stream);
    if (enqueue_closure<R>(m, k, b)) m->launches += 6;
    launch_tracer<R>(k, b, false, m->stream);
    launch_momentum<R>(k, b, false, m->stream);
    m->tend_valid = true;
}

// The reference profiles' part of the tracer totals and the wet volume: sums over the
// wet columns of (sum from the column's lowest wet level to the top of Tref dz, Sref dz,
// dz) times the column's area, in FP64 with Neumaier compensation.  They change only with
// the reference profiles, so the mixed form's reduction adds them as constants.
void reference_totals(ocean_t m) {
    double s[3] = {0.0, 0.0, 0.0}, cmp[3] = {0.0, 0.0, 0.0};
    const std::vector<double>* cols[3] = {&m->h_colT, &m->h_colS, &m->h_colV};
    for (int j = 0; j < m->ny; ++j) {
        const double ac = m->h_rows[7][j + OC_H];
        for (int i = 0; i < m->nx; ++i) {
            const int kb = m->h_kb[(size_t)(j + OC_H) * m->pitch + (i + OC_H)];
            if (kb >= m->nz) continue;
            for (int q = 0; q < 3; ++q) {
                const double x = (*cols[q])[kb] * ac, t = s[q] + x;
                cmp[q] += std::fabs(s[q]) >= std::fabs(x) ? (s[q] - t) + x : (x - t) + s[q];
                s[q] = t;
            }
        }
    }
    for (int q = 0; q < 3; ++q) m->dconst[q] = s[q] + cmp[q];
    m->dconst_ok = true;
}

template <typename R>
void enqueue_diagnostics(ocean_t m) {
    const KP<R> k = make_kp<R>(m, m->nstep == 0);
    const StepBuffers<R> b = make_bufs<R>(m);
    const size_t nr = (size_t)m->ny + 2 * OC_H;
    const int nz = m->nz;
    const double* cols = m->dlev + 4 * nz;
    DiagMetrics dm{m->drow, m->drow + nr, m->drow + 2 * nr, m->dlev, m->dlev + nz,
                   m->dlev + 2 * nz, m->dlev + 3 * nz, cols, cols + nz + 1, cols + 2 * (nz + 1),
                   m->dy, 1.0 / m->dy, m->prm.dt};
    if (sizeof(R) == sizeof(float)) {   // the mixed form's FP32 metrics and constant parts
        if (!m->dconst_ok) reference_totals(m);
        const float* rows = reinterpret_cast<const float*>(m->rowm);
        dm.fdz = m->dgf;
        dm.fdtdz = m->dgf + nz;
        dm.fAc = m->dgf + 2 * nz;
        dm.frdxc = rows + nr;
        dm.fdxv = rows + 2 * nr;
        dm.frAc = rows + 3 * nr;
        dm.fdy = (float)m->dy;
        dm.frdy = (float)(1.0 / m->dy);
        dm.fdt = (float)m->prm.dt;
        dm.cT = m->dconst[0];
        dm.cS = m->dconst[1];
        dm.cV = m->dconst[2];
    }
    launch_diagnostics<R>(k.g, dm, b.u, b.v, b.T, b.S, m->eta, m->diag_part, m->diag_out,
                          m->stream);
}

int run_diagnostics(ocean_t m, double out[8]) {
    if (m->prec == OCEAN_FP64) enqueue_diagnostics<double>(m);
    else enqueue_diagnostics<float>(m);
    OC_CUDA(m, cudaGetLastError());
    OC_CUDA(m, cudaMemcpyAsync(out, m->diag_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    OC_CUDA(m, cudaStreamSynchronize(m->stream));
    return OCEAN_OK;
}

int create_common(const ocean_grid* grid, const double* depth, const ocean_params* params,
                  void* d_arena, size_t arena_bytes, void* stream, bool own, ocean_t* out) {
    if (!out) return fail(nullptr, OCEAN_ERR_ARG, "null output handle");
    *out = nullptr;
    int rc = validate(grid, params);
    if (rc) return rc;
    if (!depth) return fail(nullptr, OCEAN_ERR_ARG, "null depth");
    ocean_t m = new ocean_s();
    configure(m, grid, params);
    const size_t need = layout(m, nullptr);
    if (own) {
        cudaError_t e = cudaMalloc(&d_arena, need);
        if (e != cudaSuccess) {
            delete m;
            return fail(nullptr, OCEAN_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", need, cudaGetErrorString(e));
        }
        arena_bytes = need;
        m->own_arena = true;
        e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaFree(d_arena);
            delete m;
            return fail(nullptr, OCEAN_ERR_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
        }
        m->own_stream = true;
    } else {
        if (!d_arena) { delete m; return fail(nullptr, OCEAN_ERR_ARG, "null arena"); }
        if (((uintptr_t)d_arena & 255) != 0) { delete m; return fail(nullptr, OCEAN_ERR_ARG, "arena must be 256-byte aligned"); }
        if (arena_bytes < need) {
            delete m;
            return fail(nullptr, OCEAN_ERR_OOM, "arena of %zu bytes is smaller than the %zu needed", arena_bytes, need);
        }
        m->stream = (cudaStream_t)stream;
    }
    m->arena = (char*)d_arena;
    m->arena_bytes = arena_bytes;
    layout(m, m->arena);
    cudaError_t e = cudaMemsetAsync(m->arena, 0, need - 256, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        int r = fail(nullptr, OCEAN_ERR_CUDA, "arena clear failed: %s", cudaGetErrorString(e));
        ocean_destroy(m);
        return r;
    }
    int se = m->prec == OCEAN_FP64 ? setup_kernel_attributes<double>(m->nz)
                                   : setup_kernel_attributes<float>(m->nz);
    if (se != 0) {
        int r = fail(nullptr, OCEAN_ERR_CUDA, "kernel attribute setup failed: %s", cudaGetErrorString((cudaError_t)se));
        ocean_destroy(m);
        return r;
    }
    if (!build_tile_maps(m)) {
        ocean_destroy(m);
        return fail(nullptr, OCEAN_ERR_CUDA, "the driver refused the tile kernels' tensor maps");
    }
    rc = build_geometry(m, depth);
    if (rc == OCEAN_OK) rc = set_wind<double>(m, params->taux, params->tauy);
    if (rc != OCEAN_OK) {
        ocean_destroy(m);
        return rc;
    }
    // state at rest with T = T0, S = S0 on wet cells
    std::vector<double> t((size_t)m->nx * m->ny * m->nz, params->T0);
    rc = ocean_set_field(m, OCEAN_T, t.data(), t.size());
    if (rc == OCEAN_OK) {
        std::fill(t.begin(), t.end(), params->S0);
        rc = ocean_set_field(m, OCEAN_S, t.data(), t.size());
    }
    if (rc == OCEAN_OK) {
        cudaError_t e2 = cudaDeviceSynchronize();
        if (e2 != cudaSuccess) rc = fail(m, OCEAN_ERR_CUDA, "create: %s", cudaGetErrorString(e2));
    }
    if (rc != OCEAN_OK) {
        ocean_destroy(m);
        return rc;
    }
    *out = m;
    return OCEAN_OK;
}

// reference profile stored-value offset of a field (T and S are kept as anomalies)
const std::vector<double>* field_reference(const ocean_t m, int id) {
    if (id == OCEAN_T) return &m->Tref;
    if (id == OCEAN_S) return &m->Sref;
    return nullptr;
}

template <typename R>
void scatter_field(const ocean_t m, const double* src, std::vector<R>& dst, bool is2d, int mask,
                   int id) {
    const std::vector<double>* ref = field_reference(m, id);
    const int nx = m->nx, ny = m->ny, nzl = is2d ? 1 : m->nz;
    dst.assign((size_t)(is2d ? m->n2pad : m->plane * m->nz), R(0));
    const std::vector<short>& kbm = mask == 1 ? m->h_kbu : mask == 2 ? m->h_kbv : m->h_kb;
    for (int k = 0; k < nzl; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long c = hix2(m, i, j);
                const bool wet = is2d ? m->h_kb[c] < m->nz : k >= kbm[c];
                const double off = ref ? (*ref)[k] : 0.0;
                dst[(size_t)k * (is2d ? 0 : m->plane) + c] =
                    wet ? (R)(src[((size_t)k * ny + j) * nx + i] - off) : R(0);
            }
}

template <typename R>
int set_field_t(ocean_t m, const FieldRef& r, int id, const double* host) {
    std::vector<R> buf;
    scatter_field<R>(m, host, buf, r.is2d, r.mask, id);
    OC_CUDA(m, cudaMemcpyAsync(r.ptr, buf.data(), buf.size() * sizeof(R), cudaMemcpyHostToDevice, m->stream));
    OC_CUDA(m, cudaStreamSynchronize(m->stream));
    return OCEAN_OK;
}

template <typename R>
int get_field_t(ocean_t m, const FieldRef& r, int id, double* host) {
    const size_t n = (size_t)(r.is2d ? m->n2pad : m->plane * m->nz);
    std::vector<R> buf(n);
    OC_CUDA(m, cudaMemcpyAsync(buf.data(), r.ptr, n * sizeof(R), cudaMemcpyDeviceToHost, m->stream));
    OC_CUDA(m, cudaStreamSynchronize(m->stream));
    const int nx = m->nx, ny = m->ny, nzl = r.is2d ? 1 : m->nz;
    std::vector<double> pref;
    if (id == OCEAN_P) pref = reference_pressure(m);
    if (id == OCEAN_T) pref = m->Tref;
    if (id == OCEAN_S) pref = m->Sref;
    const bool addref = id == OCEAN_P || id == OCEAN_T || id == OCEAN_S;
    for (int k = 0; k < nzl; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long c = hix2(m, i, j);
                double val = (double)buf[(size_t)k * (r.is2d ? 0 : m->plane) + c];
                if (addref && k >= m->h_kb[c]) val += pref[k];
                host[((size_t)k * ny + j) * nx + i] = val;
            }
    return OCEAN_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Tensor maps through the driver's entry point (no link-time dependence on libcuda).

bool oc_encode_tiled(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* ptr,
                     const unsigned long long* dims, const unsigned long long* strides,
                     const unsigned* box, CUtensorMapSwizzle swizzle) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return false;
    cuuint64_t d[5];
    cuuint64_t st[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i < rank - 1) st[i] = strides[i];
    }
    return encode(map, type, (cuuint32_t)rank, const_cast<void*>(ptr), d, st, bx, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------------------
// Model internals the batched ensemble (ocean_ensemble.cu) builds on.

int oc_member_create(const ocean_grid* grid, const double* depth, const ocean_params* params,
                     void* arena, size_t arena_bytes, void* stream, ocean_t* out) {
    return create_common(grid, depth, params, arena, arena_bytes, stream, false, out);
}

OcMemberInfo oc_member_info(const ocean_s* m) {
    OcMemberInfo r{};
    r.nx = m->nx; r.ny = m->ny; r.nz = m->nz; r.px = m->px; r.py = m->py;
    r.prec = m->prec; r.ns = m->prm.n_substeps; r.dt = m->prm.dt; r.g = m->prm.g;
    r.learned = m->prm.closure == OCEAN_CLOSURE_LEARNED || m->cl_hidden > 0;
    r.cur = m->cur; r.nstep = m->nstep;
    return r;
}

int oc_member_kb(const ocean_s* m, int i, int j) {
    return m->h_kb[hix2(const_cast<ocean_t>(m), i, j)];
}

template <typename R>
EnsMember<R> oc_member_entry(const ocean_s* m, bool first, int cur) {
    EnsMember<R> e{};
    e.k = make_kp<R>(const_cast<ocean_t>(m), first);
    e.b = make_bufs<R>(const_cast<ocean_t>(m), cur);
    const int ns = m->prm.n_substeps;
    e.dtau = (R)(2.0 * m->prm.dt / (ns + 1.0));   // as in the single-model sub-cycle
    e.rns = 1.0 / ns;
    return e;
}
template EnsMember<double> oc_member_entry<double>(const ocean_s*, bool, int);
template EnsMember<float> oc_member_entry<float>(const ocean_s*, bool, int);

void oc_member_advance(ocean_s* m) {
    m->cur = 1 - m->cur;
    m->nstep += 1;
    m->tend_valid = false;
}

// =========================================================================== C ABI

extern "C" {

int ocean_arena_bytes(const ocean_grid* grid, const ocean_params* params, size_t* bytes) {
    if (!bytes) return fail(nullptr, OCEAN_ERR_ARG, "null bytes");
    int rc = validate(grid, params);
    if (rc) return rc;
    ocean_s tmp;
    configure(&tmp, grid, params);
    *bytes = layout(&tmp, nullptr);
    return OCEAN_OK;
}

int ocean_create(const ocean_grid* grid, const double* depth, const ocean_params* params,
                 ocean_t* out) {
    return create_common(grid, depth, params, nullptr, 0, nullptr, true, out);
}

int ocean_create_in(const ocean_grid* grid, const double* depth, const ocean_params* params,
                    void* d_arena, size_t arena_bytes, void* stream, ocean_t* out) {
    return create_common(grid, depth, params, d_arena, arena_bytes, stream, false, out);
}

void ocean_destroy(ocean_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (auto& ev : h->prof_pending)
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (h->own_arena && h->arena) cudaFree(h->arena);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// message for ocean_last_error(NULL) from entry points that have no handle
void oc_set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

const char* ocean_last_error(ocean_t h) {
    return h ? h->err.c_str() : g_last_error.c_str();
}

int ocean_set_field(ocean_t h, int field, const double* host, size_t count) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!host) return fail(h, OCEAN_ERR_ARG, "null host buffer");
    FieldRef r = field_ref(h, field);
    if (!r.ptr) return fail(h, OCEAN_ERR_ARG, "unknown field id %d", field);
    if (r.readonly) return fail(h, OCEAN_ERR_ARG, "field %d is read-only", field);
    const size_t need = (size_t)h->nx * h->ny * (r.is2d ? 1 : h->nz);
    if (count != need) return fail(h, OCEAN_ERR_ARG, "field %d needs %zu values, got %zu", field, need, count);
    for (size_t q = 0; q < count; ++q)
        if (!std::isfinite(host[q])) return fail(h, OCEAN_ERR_ARG, "non-finite input value at %zu", q);
    if ((field == OCEAN_T || field == OCEAN_S) && !h->ref_locked) {
        // horizontally uniform reference profile: mean over the wet cells of each level
        std::vector<double>& ref = field == OCEAN_T ? h->Tref : h->Sref;
        const double dflt = field == OCEAN_T ? h->prm.T0 : h->prm.S0;
        for (int k = 0; k < h->nz; ++k) {
            double s = 0;
            long n = 0;
            for (int j = 0; j < h->ny; ++j)
                for (int i = 0; i < h->nx; ++i)
                    if (k >= h->h_kb[hix2(h, i, j)]) { s += host[((size_t)k * h->ny + j) * h->nx + i]; ++n; }
            ref[k] = n ? s / n : dflt;
        }
        upload_levels(h);
    }
    int rc;
    if (r.is_double) rc = set_field_t<double>(h, r, field, host);
    else if (h->prec == OCEAN_FP64) rc = set_field_t<double>(h, r, field, host);
    else rc = set_field_t<float>(h, r, field, host);
    if (rc) return rc;
    if ((h->px || h->py) && !r.is2d) {
        if (h->prec == OCEAN_FP64) {
            KP<double> k = make_kp<double>(h, true);
            double* f[1] = {reinterpret_cast<double*>(r.ptr)};
            launch_halo3<double>(k.g, f, 1, h->stream);
        } else {
            KP<float> k = make_kp<float>(h, true);
            float* f[1] = {reinterpret_cast<float*>(r.ptr)};
            launch_halo3<float>(k.g, f, 1, h->stream);
        }
        OC_CUDA(h, cudaGetLastError());
        OC_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    h->tend_valid = false;
    return OCEAN_OK;
}

int ocean_get_field(ocean_t h, int field, double* host, size_t count) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!host) return fail(h, OCEAN_ERR_ARG, "null host buffer");
    FieldRef r = field_ref(h, field);
    if (!r.ptr) return fail(h, OCEAN_ERR_ARG, "unknown field id %d", field);
    const size_t need = (size_t)h->nx * h->ny * (r.is2d ? 1 : h->nz);
    if (count != need) return fail(h, OCEAN_ERR_ARG, "field %d needs %zu values, got %zu", field, need, count);
    if (field >= OCEAN_GU && field <= OCEAN_GS && !h->tend_valid)
        return fail(h, OCEAN_ERR_STATE, "tendencies are not available: call ocean_tendencies first");
    if (r.is_double) return get_field_t<double>(h, r, field, host);
    if (h->prec == OCEAN_FP64) return get_field_t<double>(h, r, field, host);
    return get_field_t<float>(h, r, field, host);
}

int ocean_get_reference(ocean_t h, double* Tref, double* Sref) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!Tref || !Sref) return fail(h, OCEAN_ERR_ARG, "null output");
    std::copy(h->Tref.begin(), h->Tref.end(), Tref);
    std::copy(h->Sref.begin(), h->Sref.end(), Sref);
    return OCEAN_OK;
}

int ocean_set_reference(ocean_t h, const double* Tref, const double* Sref) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!Tref || !Sref) return fail(h, OCEAN_ERR_ARG, "null profile");
    for (int k = 0; k < h->nz; ++k)
        if (!std::isfinite(Tref[k]) || !std::isfinite(Sref[k]))
            return fail(h, OCEAN_ERR_ARG, "non-finite reference value at level %d", k);
    // re-express the stored anomalies against the new profiles
    const size_t n = (size_t)h->nx * h->ny * h->nz;
    std::vector<double> T(n), S(n);
    int rc = ocean_get_field(h, OCEAN_T, T.data(), n);
    if (rc == OCEAN_OK) rc = ocean_get_field(h, OCEAN_S, S.data(), n);
    if (rc) return rc;
    h->Tref.assign(Tref, Tref + h->nz);
    h->Sref.assign(Sref, Sref + h->nz);
    h->ref_locked = true;
    upload_levels(h);
    rc = ocean_set_field(h, OCEAN_T, T.data(), n);
    if (rc == OCEAN_OK) rc = ocean_set_field(h, OCEAN_S, S.data(), n);
    return rc;
}

int ocean_set_wind_stress(ocean_t h, const double* taux, const double* tauy) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    return set_wind<double>(h, taux, tauy);
}

int ocean_set_wind_stress_f32(ocean_t h, const float* taux, const float* tauy) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    return set_wind<float>(h, taux, tauy);
}

int ocean_step_async(ocean_t h, int n) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (n < 0) return fail(h, OCEAN_ERR_ARG, "n must be >= 0");
    for (int q = 0; q < n; ++q) {
        const int rc = h->prec == OCEAN_FP64 ? enqueue_step<double>(h) : enqueue_step<float>(h);
        if (rc) return rc;
    }
    OC_CUDA(h, cudaGetLastError());
    return OCEAN_OK;
}

// after a synchronisation: device waits that gave up (the learned closure's GEMM tiles,
// the tile kernels' tensor copies) become OCEAN_ERR_TIMEOUT
static int check_closure_gemm(ocean_t h) {
    if (h->cl_ready && h->prm.closure == OCEAN_CLOSURE_LEARNED && closure_gemm_failed())
        return fail(h, OCEAN_ERR_TIMEOUT, "a tensor-core GEMM tile of the closure timed out");
    if (tile_wait_failed())
        return fail(h, OCEAN_ERR_TIMEOUT, "a tile kernel's wait for its tensor copies timed out");
    return OCEAN_OK;
}

int ocean_sync(ocean_t h) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_closure_gemm(h);
}

int ocean_step(ocean_t h, int n) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (n < 0) return fail(h, OCEAN_ERR_ARG, "n must be >= 0");
    const int every = h->prm.check_every;
    for (int q = 0; q < n; ++q) {
        int rc = ocean_step_async(h, 1);
        if (rc) return rc;
        if (every > 0 && h->nstep % every == 0) {
            double d[8];
            rc = run_diagnostics(h, d);
            if (rc) return rc;
            if (d[5] != 0.0) return fail(h, OCEAN_ERR_NONFINITE, "non-finite state after step %ld", h->nstep);
            if (d[4] > 1.0) return fail(h, OCEAN_ERR_NONFINITE, "CFL number %.3g > 1 after step %ld", d[4], h->nstep);
        }
    }
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_closure_gemm(h);
}

int ocean_tendencies(ocean_t h) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (h->prec == OCEAN_FP64) enqueue_tendencies<double>(h);
    else enqueue_tendencies<float>(h);
    OC_CUDA(h, cudaGetLastError());
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    return OCEAN_OK;
}

int ocean_diagnostics(ocean_t h, ocean_diag* out) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!out) return fail(h, OCEAN_ERR_ARG, "null output");
    double d[8];
    int rc = run_diagnostics(h, d);
    if (rc) return rc;
    out->step = h->nstep;
    out->tracer_T = d[0];
    out->tracer_S = d[1];
    out->volume_eta = d[2];
    out->ke = d[3];
    out->max_cfl = d[4];
    out->nonfinite = d[5] != 0.0;
    out->wet_volume = d[6];
    return OCEAN_OK;
}

// the features' scales go to the device as reciprocals: the kernels multiply (an FP32
// division is a sequence of instructions; the BF16 features do not see the difference)
void upload_rsigma(ocean_t h, const float* sigma) {
    std::vector<float> r(6 * (size_t)h->nz);
    for (size_t q = 0; q < r.size(); ++q) r[q] = (float)(1.0 / (double)sigma[q]);
    upload_bytes(h, h->cl_sigma, r.data(), r.size() * sizeof(float));
}

int ocean_set_closure(ocean_t h, const float* params, size_t count, const float* mu,
                      const float* sigma, const ocean_closure_scales* sc) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!params || !mu || !sigma || !sc) return fail(h, OCEAN_ERR_ARG, "null argument");
    if (h->cl_hidden <= 0)
        return fail(h, OCEAN_ERR_STATE, "the model was created with closure_hidden = 0");
    if (count != ocean_mlp_param_count(h->nz, h->cl_hidden))
        return fail(h, OCEAN_ERR_ARG, "closure parameter count %zu, expected %zu", count,
                    ocean_mlp_param_count(h->nz, h->cl_hidden));
    if (closure_gemm_setup() != (int)cudaSuccess ||
        (h->prec == OCEAN_FP64 ? closure_tiles_setup<double>() : closure_tiles_setup<float>()) != (int)cudaSuccess)
        return fail(h, OCEAN_ERR_CUDA, "closure kernels' shared-memory attributes could not be set");
    const float* p = params;
    for (int l = 0; l < 4; ++l) {
        const int in = h->cl_dims[l], out = h->cl_dims[l + 1];
        upload_bytes(h, h->cl_stage, p, (size_t)in * out * sizeof(float));
        closure_weight_transpose(h->cl_stage, in, out, h->cl_Wt[l], h->stream);
        p += (size_t)in * out;
        upload_bytes(h, h->cl_b[l], p, (size_t)out * sizeof(float));
        p += out;
    }
    upload_bytes(h, h->cl_mu, mu, 6 * (size_t)h->nz * sizeof(float));
    upload_rsigma(h, sigma);
    OC_CUDA(h, cudaGetLastError());
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    h->cl_sc = *sc;
    h->cl_ready = true;
    drop_graphs(h);   // the closure's scales are launch arguments
    h->tend_valid = false;
    return OCEAN_OK;
}

int ocean_closure_features(ocean_t h, const float* mu, const float* sigma, float* d_X,
                           unsigned char* d_face, unsigned char* d_wet, float* d_dzT,
                           float* d_dzS) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (d_X && (!mu || !sigma)) return fail(h, OCEAN_ERR_ARG, "features need mu and sigma");
    if (d_X) {
        upload_bytes(h, h->cl_mu, mu, 6 * (size_t)h->nz * sizeof(float));
        upload_rsigma(h, sigma);
    }
    if (h->prec == OCEAN_FP64) {
        const KP<double> k = make_kp<double>(h, false);
        const StepBuffers<double> b = make_bufs<double>(h);
        launch_closure_features<double>(k, b.u, b.v, b.T, b.S, h->cl_mu, h->cl_sigma, d_X, nullptr,
                                        d_face, d_wet, d_dzT, d_dzS, h->stream);
    } else {
        const KP<float> k = make_kp<float>(h, false);
        const StepBuffers<float> b = make_bufs<float>(h);
        launch_closure_features<float>(k, b.u, b.v, b.T, b.S, h->cl_mu, h->cl_sigma, d_X, nullptr,
                                       d_face, d_wet, d_dzT, d_dzS, h->stream);
    }
    h->launches += 1;
    OC_CUDA(h, cudaGetLastError());
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    return OCEAN_OK;
}

int ocean_coarse_grain(ocean_t f, ocean_t c, int r, float* d_FT, float* d_FS, float* d_GTm,
                       float* d_GSm) {
    if (!f || !c) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!d_FT || !d_FS || !d_GTm || !d_GSm) return fail(f, OCEAN_ERR_ARG, "null output");
    if (r < 1 || c->nx * r != f->nx || c->ny * r != f->ny || c->nz != f->nz || c->prec != f->prec ||
        c->px != f->px || c->py != f->py)
        return fail(f, OCEAN_ERR_ARG, "coarse grid must be the fine grid with nx, ny divided by r");
    for (int k = 0; k <= f->nz; ++k)
        if (f->zf[k] != c->zf[k]) return fail(f, OCEAN_ERR_ARG, "fine and coarse levels differ");
    if (f->Tref != c->Tref || f->Sref != c->Sref)
        return fail(f, OCEAN_ERR_ARG, "fine and coarse reference profiles differ (ocean_set_reference)");
    if (!f->tend_valid) return fail(f, OCEAN_ERR_STATE, "call ocean_tendencies on the fine model first");
    OC_CUDA(f, cudaStreamSynchronize(c->stream));
    const int fc = f->cur, fn = 1 - f->cur, cc = c->cur;
    if (f->prec == OCEAN_FP64) {
        using R = double;
        auto P = [](void* q) { return reinterpret_cast<R*>(q); };
        const KP<R> kf = make_kp<R>(f, false), kc = make_kp<R>(c, false);
        launch_coarse_grain<R>(kf, kc, r, P(f->u[fc]), P(f->v[fc]), P(f->T[fc]), P(f->S[fc]), P(f->w),
                               P(f->T[fn]), P(f->S[fn]), f->eta, P(c->u[cc]), P(c->v[cc]),
                               P(c->T[cc]), P(c->S[cc]), c->eta, d_FT, d_FS, d_GTm, d_GSm, f->stream);
        if (c->px || c->py) {
            R* q[4] = {P(c->u[cc]), P(c->v[cc]), P(c->T[cc]), P(c->S[cc])};
            launch_halo3<R>(kc.g, q, 4, f->stream);
        }
    } else {
        using R = float;
        auto P = [](void* q) { return reinterpret_cast<R*>(q); };
        const KP<R> kf = make_kp<R>(f, false), kc = make_kp<R>(c, false);
        launch_coarse_grain<R>(kf, kc, r, P(f->u[fc]), P(f->v[fc]), P(f->T[fc]), P(f->S[fc]), P(f->w),
                               P(f->T[fn]), P(f->S[fn]), f->eta, P(c->u[cc]), P(c->v[cc]),
                               P(c->T[cc]), P(c->S[cc]), c->eta, d_FT, d_FS, d_GTm, d_GSm, f->stream);
        if (c->px || c->py) {
            R* q[4] = {P(c->u[cc]), P(c->v[cc]), P(c->T[cc]), P(c->S[cc])};
            launch_halo3<R>(kc.g, q, 4, f->stream);
        }
    }
    f->launches += 2;
    OC_CUDA(f, cudaGetLastError());
    OC_CUDA(f, cudaStreamSynchronize(f->stream));
    c->tend_valid = false;
    return OCEAN_OK;
}

int ocean_closure_targets(ocean_t c, const float* d_GTm, const float* d_GSm, const float* d_FT,
                          const float* d_FS, float* d_GTt, float* d_GSt) {
    if (!c) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!d_GTm || !d_GSm || !d_FT || !d_FS || !d_GTt || !d_GSt)
        return fail(c, OCEAN_ERR_ARG, "null device array");
    if (!c->tend_valid) return fail(c, OCEAN_ERR_STATE, "call ocean_tendencies on the coarse model first");
    const int n = 1 - c->cur;
    if (c->prec == OCEAN_FP64) {
        const KP<double> k = make_kp<double>(c, false);
        launch_closure_targets<double>(k, reinterpret_cast<double*>(c->T[n]),
                                       reinterpret_cast<double*>(c->S[n]), d_GTm, d_GSm, d_FT,
                                       d_FS, d_GTt, d_GSt, c->stream);
    } else {
        const KP<float> k = make_kp<float>(c, false);
        launch_closure_targets<float>(k, reinterpret_cast<float*>(c->T[n]),
                                      reinterpret_cast<float*>(c->S[n]), d_GTm, d_GSm, d_FT, d_FS,
                                      d_GTt, d_GSt, c->stream);
    }
    c->launches += 1;
    OC_CUDA(c, cudaGetLastError());
    OC_CUDA(c, cudaStreamSynchronize(c->stream));
    return OCEAN_OK;
}

int ocean_profile(ocean_t h, int enable) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto& ev : h->prof_pending)
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    h->prof_pending.clear();
    if (enable) {
        for (double& x : h->phase_ms) x = 0.0;
        h->prof_steps = 0;
    }
    h->prof = enable != 0;
    return OCEAN_OK;
}

int ocean_phase_times(ocean_t h, double* ms, int n, long* steps) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (!ms || n < 0) return fail(h, OCEAN_ERR_ARG, "bad output");
    OC_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto& ev : h->prof_pending) {
        for (size_t q = 0; q + 1 < ev.size() && q < OCEAN_NPHASE; ++q) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
            h->phase_ms[q] += t;
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        h->prof_steps += 1;
    }
    h->prof_pending.clear();
    for (int q = 0; q < n && q < OCEAN_NPHASE; ++q) ms[q] = h->phase_ms[q];
    if (steps) *steps = h->prof_steps;
    return OCEAN_OK;
}

long ocean_kernel_launches(ocean_t h) { return h ? h->launches : -1; }

long ocean_get_step(ocean_t h) { return h ? h->nstep : -1; }

int ocean_set_step(ocean_t h, long step) {
    if (!h) return fail(nullptr, OCEAN_ERR_ARG, "null handle");
    if (step < 0) return fail(h, OCEAN_ERR_ARG, "step must be >= 0");
    h->nstep = step;
    return OCEAN_OK;
}

void* ocean_stream(ocean_t h) { return h ? (void*)h->stream : nullptr; }

}  // extern "C"
