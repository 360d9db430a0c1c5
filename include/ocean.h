/*
 * ocean.h -- C ABI of the GB300 hydrostatic free-surface ocean step (libocean.so).
 *
 * The library advances one explicit baroclinic time step of the hydrostatic
 * Boussinesq equations on an Arakawa C-grid (arXiv 2309.06662, Sec. "New numerical
 * methods for finite volume fluid dynamics on the sphere": finite volumes on a
 * staggered C-grid, implicit-explicit second-order Adams-Bashforth stepping,
 * backward-Euler vertical diffusion with a tridiagonal solve, adaptive-order WENO
 * advection of momentum and tracers; Sec. "Optimization of ocean free surface
 * dynamics": split-explicit barotropic sub-cycling; Sec. "How performance was
 * measured": Richardson-number vertical mixing, no explicit horizontal diffusion).
 * Every step runs in CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every call:
 *  - Return codes: OCEAN_OK (0) or a negative OCEAN_ERR_* code; the message is
 *    available from ocean_last_error(handle) (or ocean_last_error(NULL) when no
 *    handle exists yet).  No C++ exception crosses this boundary.
 *  - Indexing: i is the zonal (x) index, j the meridional (y) index, k the level;
 *    k = 0 is the BOTTOM level, k = nz-1 the top.  3-D host arrays are [nz][ny][nx]
 *    (i fastest), 2-D host arrays [ny][nx].  No halo on the host side.
 *  - Staggering: u(i,j,k) lives on the west face of cell (i,j,k), v(i,j,k) on its
 *    south face, w(i,j,k) on its bottom face, T, S, p at the cell centre; kappa and
 *    nu on the bottom (w-)face.
 *  - Host arrays cross the ABI as double, whatever the internal precision.  Values on
 *    dry cells/faces are ignored on input and returned as 0.
 *  - Ownership: the library copies every host input; the caller owns its buffers.
 *    Device memory belongs to the handle (or to the caller, with ocean_create_in).
 *  - Threads: a handle is not thread-safe; distinct handles are independent.
 */
#ifndef OCEAN_H
#define OCEAN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCEAN_OK 0
#define OCEAN_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, bad id) */
#define OCEAN_ERR_CUDA (-2)      /* a CUDA call failed */
#define OCEAN_ERR_NONFINITE (-3) /* the health check found a NaN/Inf or CFL > 1 */
#define OCEAN_ERR_TIMEOUT (-4)   /* a bounded device wait gave up */
#define OCEAN_ERR_OOM (-5)       /* device allocation failed or arena too small */
#define OCEAN_ERR_STATE (-6)     /* call not valid in the handle's current state */

#define OCEAN_FP64 0             /* every field and stencil in FP64 */
#define OCEAN_MIXED 1            /* FP32 fields and stencils, FP64 free surface and
                                    conservation sums */

#define OCEAN_CLOSURE_RI 0       /* Richardson-number closure */
#define OCEAN_CLOSURE_LEARNED 1  /* column MLP, with the Ri closure as fallback */

/* field ids for ocean_set_field / ocean_get_field */
#define OCEAN_U 0
#define OCEAN_V 1
#define OCEAN_T 2
#define OCEAN_S 3
#define OCEAN_ETA 4        /* 2-D free-surface height, m */
#define OCEAN_GU_PREV 5    /* tendencies of the last completed step (AB2 memory) */
#define OCEAN_GV_PREV 6
#define OCEAN_GT_PREV 7
#define OCEAN_GS_PREV 8
#define OCEAN_W 9          /* diagnostics of the last ocean_tendencies call (read only) */
#define OCEAN_P 10
#define OCEAN_KAPPA 11
#define OCEAN_NU 12
#define OCEAN_GU 13        /* tendencies G^n of the last ocean_tendencies call (read only) */
#define OCEAN_GV 14
#define OCEAN_GT 15
#define OCEAN_GS 16
#define OCEAN_HU 17        /* 2-D depth of the u- and v-columns (read only) */
#define OCEAN_HV 18
#define OCEAN_T_ANOM 19    /* the stored anomalies T - Tref(k), S - Sref(k): what a bitwise */
#define OCEAN_S_ANOM 20    /* checkpoint saves (with the profiles of ocean_get_reference) */

typedef struct ocean_s* ocean_t;

/* Grid.  kind 0: Cartesian beta-plane, x0..x1 and y0..y1 in metres.  kind 1: latitude-
 * longitude, x0..x1 longitude and y0..y1 latitude in degrees.  z_faces holds nz+1
 * level faces, increasing from the sea floor (-H) to the surface (0); copied. */
typedef struct {
    int kind;
    int nx, ny, nz;
    int periodic_x, periodic_y;
    double x0, x1, y0, y1;
    const double* z_faces;
} ocean_grid;

/* Parameters.  taux/tauy: surface wind stress on u-/v-faces, [ny][nx], N/m^2; copied
 * (NULL = no wind).  check_every: run the non-finite/CFL health check every that many
 * steps inside ocean_step (0 = never). */
typedef struct {
    double dt;              /* baroclinic time step, s */
    int n_substeps;         /* barotropic substeps N_s >= 1 */
    double chi;             /* quasi-AB2 offset (0.1) */
    double g, rho0;         /* gravity, reference density */
    double alpha, beta_s;   /* linear EOS: b = g[alpha (T - T0) - beta_s (S - S0)] */
    double T0, S0;
    double f0, beta_plane;  /* Cartesian Coriolis f = f0 + beta (y - (y0+y1)/2) */
    double omega, radius;   /* lat-lon: f = 2 omega sin(phi), planet radius */
    double nu0, ri_a, nu_b, kappa_b, kappa_conv; /* Richardson-number closure */
    double weno_eps;        /* WENO-Z epsilon */
    int weno_linear;        /* 1: ideal (linear) weights, a test switch */
    double min_depth;       /* columns shallower than this are land, m */
    int precision;          /* OCEAN_FP64 or OCEAN_MIXED */
    int closure;            /* OCEAN_CLOSURE_RI or OCEAN_CLOSURE_LEARNED */
    int check_every;
    const double* taux;
    const double* tauy;
    int closure_hidden;     /* hidden width of the learned closure to reserve memory for
                               (0 = none; otherwise a multiple of 16) */
    int baro_filter;        /* time average closing the barotropic sub-cycle:
                               OCEAN_FILTER_BOXCAR or OCEAN_FILTER_POWER_LAW */
    int vertical_weno;      /* coefficients of the vertical WENO reconstructions:
                               OCEAN_VWENO_INDEX or OCEAN_VWENO_STRETCHED */
    int momentum_vadv;      /* vertical momentum advection: OCEAN_VADV_CENTRED or
                               OCEAN_VADV_WENO */
} ocean_params;

/* Averaging filters of the split-explicit sub-cycle (Sec. "Optimization of ocean free
 * surface dynamics": the fast mode is sub-cycled and averaged back onto the baroclinic
 * step).  Both are weights a_1..a_Ns with sum 1; the substep is dtau = dt / sum_m m a_m,
 * which puts the average's centroid at t + dt.  BOXCAR: a_m = 1/Ns (dtau = 2 dt/(Ns+1)).
 * POWER_LAW: the shape x^2 (1 - x^4) - 0.284 x of Shchepetkin & McWilliams (2005) over its
 * support (0, xs), sampled at m xs/(Ns+1) and normalised (a short negative lobe, then one
 * positive lobe; it damps the unresolved fast modes more than the boxcar). */
#define OCEAN_FILTER_BOXCAR 0
#define OCEAN_FILTER_POWER_LAW 1

/* Vertical reconstructions on stretched levels (the adaptive WENO of Sec. "New numerical
 * methods for finite volume fluid dynamics on the sphere" on a non-uniform grid).  INDEX:
 * the uniform-grid coefficients in level index space.  STRETCHED: the candidate
 * polynomials and ideal weights of each level face from the actual level thicknesses
 * (fifth order on smoothly stretched levels); the smoothness indicators keep their
 * index-space form.  Applies to the vertical tracer fluxes and, with OCEAN_VADV_WENO, to
 * the vertical momentum advection. */
#define OCEAN_VWENO_INDEX 0
#define OCEAN_VWENO_STRETCHED 1

/* Vertical advection term w du/dz of the vector-invariant momentum equation (Sec. "New
 * numerical methods for finite volume fluid dynamics on the sphere").  CENTRED:
 * 1/2 [w_top (u_{k+1} - u_k)/dzf_{k+1} + w_bot (u_k - u_{k-1})/dzf_k].  WENO: the flux form
 * [w_top u~_top - w_bot u~_bot - u_k (w_top - w_bot)] / dz_k with u~ the upwind WENO
 * reconstruction at the level faces (adaptive order at the column ends).  w at a u-face is
 * the mean of the two neighbouring columns' w; no flux through the surface or below the
 * face's lowest wet level.  The batched ensemble runs the defaults (INDEX, CENTRED). */
#define OCEAN_VADV_CENTRED 0
#define OCEAN_VADV_WENO 1

typedef struct {
    long step;              /* completed steps */
    double tracer_T;        /* sum T dV over wet cells (compensated FP64) */
    double tracer_S;        /* sum S dV */
    double volume_eta;      /* sum eta dA over wet columns */
    double ke;              /* 1/2 sum u^2 dV_u + 1/2 sum v^2 dV_v */
    double max_cfl;         /* max advective CFL number |u| dt/dx, |v| dt/dy, |w| dt/dz */
    double wet_volume;      /* sum dV over wet cells */
    int nonfinite;          /* 1 if any prognostic value is NaN/Inf */
} ocean_diag;

/* Device bytes ocean_create_in needs for this grid and these parameters. */
int ocean_arena_bytes(const ocean_grid* grid, const ocean_params* params, size_t* bytes);

/* Build a model: validates the grid, builds metrics and masks from depth ([ny][nx], m,
 * >= 0; copied), allocates its device memory with cudaMalloc on the current device and
 * creates its own stream.  State starts at rest: u = v = eta = 0, T = T0, S = S0. */
int ocean_create(const ocean_grid* grid, const double* depth, const ocean_params* params,
                 ocean_t* out);

/* As ocean_create, but inside caller-owned device memory d_arena (at least
 * ocean_arena_bytes, 256-byte aligned) and on the caller's cudaStream_t `stream` (NULL =
 * legacy default stream).  The caller keeps the memory alive until ocean_destroy. */
int ocean_create_in(const ocean_grid* grid, const double* depth, const ocean_params* params,
                    void* d_arena, size_t arena_bytes, void* stream, ocean_t* out);

void ocean_destroy(ocean_t h);
const char* ocean_last_error(ocean_t h);

/* Copy a host field in (count must equal the field's element count) or out.  Setting
 * u or v leaves the AB2 memory alone; setting T or S also resets the horizontally
 * uniform reference profiles the library subtracts before the pressure integral. */
int ocean_set_field(ocean_t h, int field, const double* host, size_t count);
int ocean_get_field(ocean_t h, int field, double* host, size_t count);

/* The horizontally uniform reference profiles Tref[k], Sref[k] (nz values each, host).
 * The library stores T and S as anomalies from them (in the mixed form this keeps the
 * buoyancy resolution that drives the horizontal pressure gradient).  By default
 * ocean_set_field(T or S) resets the profile to the mean of the given field over the wet
 * cells of each level; after ocean_set_reference the profiles stay fixed, and the stored
 * state is re-expressed so that T and S themselves do not change.  A checkpoint that
 * saves the profiles and restores them before the fields resumes bit for bit. */
int ocean_get_reference(ocean_t h, double* Tref, double* Sref);
int ocean_set_reference(ocean_t h, const double* Tref, const double* Sref);

/* Replace the surface wind stress (host arrays [ny][nx] in N/m^2, either may be NULL for
 * zero).  The arrays are copied to a staging area of the model's device memory on the
 * model's stream, after the work already enqueued there, and scaled into the model's
 * fields by a kernel; the call returns once the copies have completed, so the caller may
 * reuse the arrays at once.  Errors: OCEAN_ERR_ARG (null handle), OCEAN_ERR_CUDA. */
int ocean_set_wind_stress(ocean_t h, const double* taux, const double* tauy);

/* The same from FP32 host arrays: half the bytes over the host link.  Each value is
 * widened to FP64 before the scaling, so a float array gives the fields that the double
 * array of the same values gives (in either precision of the model; an FP64 model then
 * sees the float values).  Errors: OCEAN_ERR_ARG (null handle), OCEAN_ERR_CUDA. */
int ocean_set_wind_stress_f32(ocean_t h, const float* taux, const float* tauy);

/* Advance n >= 0 steps and wait for them; runs the health check when check_every > 0.
 * One step n -> n+1 is the sequence of the paper's Sec. "New numerical methods for finite
 * volume fluid dynamics on the sphere" and Sec. "Optimization of ocean free surface
 * dynamics": the pressure and vertical-diffusivity intermediates of the state at n (Sec.
 * "Starting from scratch with Julia"), WENO tracer and vector-invariant momentum
 * tendencies, the quasi-second-order Adams-Bashforth predictor, backward-Euler vertical
 * diffusion (one tridiagonal solve per column), the split-explicit barotropic sub-cycle
 * with its time-averaging filter, and the barotropic correction of u, v.  The first step
 * of a model (step counter 0) is forward Euler.  Errors: OCEAN_ERR_ARG (null handle,
 * n < 0), OCEAN_ERR_CUDA, OCEAN_ERR_NONFINITE (health check), OCEAN_ERR_TIMEOUT (a
 * bounded device wait gave up). */
int ocean_step(ocean_t h, int n);

/* Enqueue n steps on the handle's stream and return without waiting. */
int ocean_step_async(ocean_t h, int n);

/* Wait for all work queued on the handle's stream. */
int ocean_sync(ocean_t h);

/* Compute the diagnostics (w, p, kappa, nu) and the tendencies G^n of the current
 * state without stepping (fields OCEAN_W .. OCEAN_GS). */
int ocean_tendencies(ocean_t h);

/* Conservation and health diagnostics of the current state (synchronous).  The paper
 * measures conservation only implicitly (its runs are long and stable, Sec. "How
 * performance was measured"); these sums are the check that a finite-volume step in
 * flux form with a closed basin keeps sum T dV, sum S dV and sum eta dA fixed to
 * roundoff.  Total tracer
 * contents and volume (compensated FP64 over columns), kinetic energy, the largest
 * advective CFL number (w integrated from the current u, v inside the same reduction,
 * so the fields OCEAN_W .. OCEAN_NU are left as the last ocean_tendencies or step made
 * them), and whether any state value is not finite.  Errors: OCEAN_ERR_ARG (null
 * arguments), OCEAN_ERR_CUDA. */
int ocean_diagnostics(ocean_t h, ocean_diag* out);

long ocean_get_step(ocean_t h);
int ocean_set_step(ocean_t h, long step);

/* The handle's stream (a cudaStream_t). */
void* ocean_stream(ocean_t h);

/* Per-phase timing of ocean_step: with profiling on, every step records CUDA events on
 * the handle's stream between its phases.  enable = 1 clears the totals and starts,
 * 0 stops (both wait for queued work).  ocean_phase_times waits for the stream and
 * returns in ms[0..n) the summed device time of each phase over the steps timed so far
 * (*steps).  Phases: */
#define OCEAN_PHASE_DIAG 0         /* pressure, w, Richardson-number closure */
#define OCEAN_PHASE_TRACER 1       /* T, S tendencies + AB2 + vertical diffusion */
#define OCEAN_PHASE_MOMENTUM 2     /* u, v tendencies + AB2 + vertical viscosity */
#define OCEAN_PHASE_BAROTROPIC 3   /* split-explicit sub-cycle and averaging */
#define OCEAN_PHASE_CORRECT 4      /* barotropic correction and halo copies */
#define OCEAN_NPHASE 5
int ocean_profile(ocean_t h, int enable);
int ocean_phase_times(ocean_t h, double* ms, int n, long* steps);

/* Number of kernels this handle has enqueued so far (all entry points). */
long ocean_kernel_launches(ocean_t h);

/* ---- component entry points (device pointers, caller-owned, on `stream`) ---- */

/* Adaptive-order WENO-Z reconstruction on a periodic 1-D row (Sec. "New numerical
 * methods", adaptive-order WENO): for each face f in [0, n) between cells f-1 and f,
 * out[f] = reconstruction upwind by the sign of vel[f] (vel >= 0 takes cell f-1 as the
 * upwind cell), using the fifth-order stencil when all five cells have inside[] != 0,
 * else the third-order one, else the upwind value.  q, vel, out: n values of the given
 * precision (double for OCEAN_FP64, float for OCEAN_MIXED); inside: n bytes (NULL =
 * all inside). */
int ocean_weno_faces(const void* d_q, const void* d_vel, const unsigned char* d_inside, int n,
                     void* d_out, int precision, double eps, int linear, void* stream);

/* Batched tridiagonal solve (Sec. "New numerical methods": backward Euler + tridiagonal
 * solver): for each of nsys systems s, a[k] x[k-1] + b[k] x[k] + c[k] x[k+1] = d[k],
 * k = 0..n-1 (a[0], c[n-1] ignored), by the Thomas algorithm without pivoting (the
 * caller guarantees diagonal dominance).  Arrays are level-major: element (k, s) at
 * k*nsys + s, of the given precision.  1 <= n <= 256. */
int ocean_tridiag_batched(const void* d_a, const void* d_b, const void* d_c, const void* d_d,
                          void* d_x, int n, int nsys, int precision, void* stream);

/* ---- learned column closure (the network, its loss and its training) ----
 *
 * A column MLP standing in for the subgrid tracer fluxes (the paper's own runs use the
 * Richardson-number closure, Sec. "How performance was measured"; this network is an
 * extension trained on coarse-grained fine runs of this same solver).  Layers:
 * x (6 nz) -> H -> H -> H -> y (3 nz), SiLU after each hidden layer, BF16 tensor-core
 * GEMMs with FP32 accumulation and FP32 master weights.  Inputs per column: T, S,
 * centre-averaged u, v at the nz levels, N^2 and shear^2 on the nz bottom faces, each
 * z-scored, 0 on dry levels.  Outputs: kappa_k = kappa softplus(y_k) (vertical
 * diffusivity on face k, added to the Richardson-number one), dG_T = gT y_{nz+k}, dG_S = gS y_{2nz+k} (tracer tendency
 * corrections).  Flat parameter layout: for each layer W [in][out] row-major, then b
 * [out]. */
typedef struct ocean_mlp_s* ocean_mlp_t;

/* Device pointers of one training batch of M columns: X [M][6nz] normalised features
 * (fp32); per face or level [M][nz]: dzT, dzS (coarse vertical gradients on faces), FT,
 * FS (subgrid vertical fluxes on faces), GT, GS (lateral residual tendencies on levels);
 * face, wet (1 = the entry counts). */
typedef struct {
    const float *X, *dzT, *dzS, *FT, *FS, *GT, *GS;
    const unsigned char *face, *wet;
} ocean_batch;

/* Output scales and loss normalisations:
 * L = mean_face[((-kappa_k dzT - FT)/sFT)^2 + ((-kappa_k dzS - FS)/sFS)^2]
 *   + mean_wet[((dG_T - GT)/sGT)^2 + ((dG_S - GS)/sGS)^2]. */
typedef struct {
    float kappa, gT, gS, sFT, sFS, sGT, sGS;
} ocean_closure_scales;

size_t ocean_mlp_param_count(int nz, int hidden);
/* Allocates the weights, Adam state and activations for batches of up to max_batch
 * columns (a multiple of 8) on `stream`; params may be NULL (zeros). */
int ocean_mlp_create(int nz, int hidden, int max_batch, const float* params, void* stream,
                     ocean_mlp_t* out);
void ocean_mlp_destroy(ocean_mlp_t h);
int ocean_mlp_set_params(ocean_mlp_t h, const float* host, size_t count);  /* resets Adam */
int ocean_mlp_get_params(ocean_mlp_t h, float* host, size_t count);
/* y = MLP(x) for M <= max_batch rows: d_X fp32 [M][6nz], d_Y fp32 [M][3nz] */
int ocean_mlp_forward(ocean_mlp_t h, const float* d_X, int M, float* d_Y);
/* The same from BF16 inputs d_Xb [M][6nz] (16-byte aligned), as the model's step feeds the
 * network: no conversion, only the four GEMMs and their epilogues. */
int ocean_mlp_forward_bf16(ocean_mlp_t h, const void* d_Xb, int M, float* d_Y);
/* Loss of a batch and the gradients (to host_grads in the flat layout, if not NULL). */
int ocean_mlp_loss_grad(ocean_mlp_t h, const ocean_batch* batch, int M,
                        const ocean_closure_scales* scales, float* loss, float* host_grads);
/* One Adam step (lr; beta = 0.9, 0.999; eps = 1e-8) on a batch; the loss before it. */
int ocean_mlp_train_step(ocean_mlp_t h, const ocean_batch* batch, int M,
                         const ocean_closure_scales* scales, float lr, float* loss);

/* Self-test of the bounded device waits the tensor-core GEMMs use (a wait on an mbarrier
 * that gives up after ~1 s and reports OCEAN_ERR_TIMEOUT instead of hanging the GPU): one
 * kernel on `stream` waits on a barrier that nothing completes, with a limit of `cycles`
 * SM clock cycles.  Returns OCEAN_ERR_TIMEOUT when the wait gave up (the expected
 * outcome; the CUDA context stays usable), OCEAN_OK if the barrier completed. */
int ocean_selftest_bounded_wait(long long cycles, void* stream);

/* Load a trained closure into a model created with closure_hidden > 0: the flat network
 * parameters (ocean_mlp_param_count(nz, closure_hidden) floats), the feature statistics
 * mu, sigma (6 nz each, host) and the output scales.  From then on every step with
 * params.closure == OCEAN_CLOSURE_LEARNED runs the network on all columns after the
 * Richardson-number closure: its diffusivity is added to kappa on the interior wet faces
 * and its corrections to the tracer tendencies; a column with any non-finite output keeps
 * the Richardson-number kappa alone and gets no correction. */
int ocean_set_closure(ocean_t h, const float* params, size_t count, const float* mu,
                      const float* sigma, const ocean_closure_scales* scales);

/* Network inputs of the model's current state for every column c = j nx + i (device
 * outputs, each may be NULL): d_X [nx ny][6nz] z-scored with mu, sigma (host, 6nz each;
 * required with d_X), d_face / d_wet [nx ny][nz] masks (interior wet faces, wet levels),
 * d_dzT / d_dzS [nx ny][nz] vertical gradients of T and S on the faces. */
int ocean_closure_features(ocean_t h, const float* mu, const float* sigma, float* d_X,
                           unsigned char* d_face, unsigned char* d_wet, float* d_dzT,
                           float* d_dzS);

/* Coarse-grain the fine model's state onto the coarse one (same levels, same reference
 * profiles, nx and ny r times smaller): tracers and the fine tendencies of the last
 * ocean_tendencies call as volume means over wet fine cells, u and v as means over the
 * wet fine faces on each coarse face, eta as an area mean.  The coarse state is replaced
 * (its step count is left alone).  Device outputs [ncoarse][nz]: d_FT, d_FS the subgrid
 * vertical fluxes <w T_f> - <w><T_f> on coarse faces, d_GTm, d_GSm the mean fine
 * tendencies. */
int ocean_coarse_grain(ocean_t fine, ocean_t coarse, int r, float* d_FT, float* d_FS,
                       float* d_GTm, float* d_GSm);

/* Lateral residual targets on the coarse model (after ocean_tendencies on it):
 * d_GTt = d_GTm - G_T(coarse) + (F_{k+1} - F_k)/dz_k, and likewise for S. */
int ocean_closure_targets(ocean_t coarse, const float* d_GTm, const float* d_GSm,
                          const float* d_FT, const float* d_FS, float* d_GTt, float* d_GSt);

/* The batched tridiagonal solve above, for callers that cannot allocate device memory:
 * code embedded in a host framework whose caching allocator owns the device's free
 * memory (a cudaMalloc of ours could fail, or fragment its pool), a runtime with a fixed
 * memory budget set at start-up, or a latency-bound loop that must not make the
 * device-synchronising cudaMalloc/cudaFree calls.  It allocates nothing: the Thomas coefficients go to one
 * static device array of OCEAN_TRIDIAG_STATIC_WORDS 8-byte words (16 MiB) that every GPU
 * loading the library holds until the process exits.  Same arguments, layout and result
 * as ocean_tridiag_batched, with n >= 1 and n * nsys at most OCEAN_TRIDIAG_STATIC_WORDS
 * (OCEAN_FP64) or twice that (OCEAN_MIXED); larger requests return OCEAN_ERR_ARG with a
 * message and launch nothing.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) while that device is current and keeps it for the
 * life of the process; make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) invalidates the kept address: later calls in the same process are
 * then invalid.  All calls share the array and it keeps the last call's
 * contents (nothing needs clearing: every value read is first written by the same
 * call); calls that overlap on the GPU race on it.  The paper has no counterpart. */
#define OCEAN_TRIDIAG_STATIC_WORDS (1 << 21)
int ocean_tridiag_batched_static(const void* d_a, const void* d_b, const void* d_c,
                                 const void* d_d, void* d_x, int n, int nsys, int precision,
                                 void* stream);

/* ---- batched ensemble ----
 *
 * Many independent models (members) of different sizes advanced together: one step of
 * the ensemble is one step of every member, run as one sequence of persistent kernels
 * whose blocks take work items (member, column chunk / tile / barotropic region) from a
 * list sorted by decreasing cost, so that one launch per phase covers all members (the
 * paper motivates ensembles in its introduction but runs none; this is this library's
 * design).  After the first step each step is one CUDA graph launch.  Each member
 * computes what ocean_step computes for it alone, to rounding (the ensemble kernels are a
 * second compiled instance of the same kernel bodies and may fuse multiply-adds
 * differently); the choice of launch shapes never changes a bit.
 *
 * Members are created from per-member grids, depths and parameters (arrays of length
 * `members`) in one device allocation on one stream owned by the ensemble; they must
 * share precision, dt and n_substeps, be closed (no periodic direction) and use the
 * Richardson-number closure.  ocean_ensemble_member returns a member's handle (owned by
 * the ensemble; do not destroy it): ocean_set_field, ocean_get_field, ocean_diagnostics
 * and the other per-model calls work on it.  Stepping a member on its own with
 * ocean_step puts it out of step with the others; ocean_ensemble_step then returns
 * OCEAN_ERR_STATE until all members have taken the same number of steps again. */
typedef struct ocean_ensemble_s* ocean_ensemble_t;
int ocean_ensemble_create(int members, const ocean_grid* grids, const double* const* depths,
                          const ocean_params* params, ocean_ensemble_t* out);
void ocean_ensemble_destroy(ocean_ensemble_t e);
int ocean_ensemble_size(ocean_ensemble_t e);
ocean_t ocean_ensemble_member(ocean_ensemble_t e, int i);     /* NULL if out of range */
void* ocean_ensemble_stream(ocean_ensemble_t e);              /* cudaStream_t */
/* n steps of every member; _async returns once they are enqueued */
int ocean_ensemble_step(ocean_ensemble_t e, int n);
int ocean_ensemble_step_async(ocean_ensemble_t e, int n);
/* Autotuner of the launch shapes: runs reps x (largest candidate count) real steps (they
 * advance the ensemble; every candidate computes the same result), timing each kernel
 * kind under each candidate grid size (one item per block, or persistent with 1, 2 or
 * the occupancy limit of blocks per SM) and schedule (static or atomic counter), then
 * keeps the fastest per kind and rebuilds the step graphs.  *steps_taken receives the
 * number of steps run (may be NULL). */
int ocean_ensemble_autotune(ocean_ensemble_t e, int reps, int* steps_taken);
/* Autotuner of the barotropic region shape, the one-GPU form of the paper's barotropic
 * halo as wide as the sub-cycle (Sec. "Optimization of ocean free surface dynamics"): a
 * region of 64 x 32 columns advances bs substeps per pass over HBM, with a halo of bs
 * columns, so a wider halo means fewer passes but a smaller interior.  For each bs of 4, 6
 * and 8 it runs reps real steps (they advance the ensemble) and times the sub-cycle's
 * passes, then keeps the fastest and rebuilds the step graphs.  Results under different bs
 * agree to rounding (the FP32 partial averages of a pass are added into the FP64
 * accumulators once per pass), not bit for bit.  *steps_taken may be NULL. */
int ocean_ensemble_autotune_regions(ocean_ensemble_t e, int reps, int* steps_taken);
/* The halo width (substeps per pass) in use; set it to 4, 6 or 8 (OCEAN_ERR_ARG
 * otherwise).  The default is 6, the single model's. */
int ocean_ensemble_region_substeps(ocean_ensemble_t e);
int ocean_ensemble_set_region_substeps(ocean_ensemble_t e, int bs);
/* Best sub-cycle time (ms per step) the region autotuner measured for bs = 4, 6, 8 (three
 * floats; 0 before tuning). */
int ocean_ensemble_region_times(ocean_ensemble_t e, float* ms);
/* Launch shape of each kernel kind (OCEAN_ENS_NKIND entries each): blocks per launch,
 * 1 if the atomic-counter schedule is used, and the number of work items. */
#define OCEAN_ENS_NKIND 7   /* diag, tracer, momentum, baro begin, baro pass, baro end, correct */
int ocean_ensemble_launch_shapes(ocean_ensemble_t e, int* grid, int* dynamic, int* items);
/* kernels enqueued by the ensemble's own steps */
long ocean_ensemble_kernel_launches(ocean_ensemble_t e);
/* Device time (ms, CUDA events on the ensemble's stream) of each kernel kind's launches
 * in one step under its chosen shape, the best over the autotuner's steps (all passes
 * together for the barotropic pass); 0 before ocean_ensemble_autotune. */
int ocean_ensemble_kind_times(ocean_ensemble_t e, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* OCEAN_H */
