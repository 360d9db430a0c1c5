// ocean_ensemble.cu -- host side of the batched ensemble: members in one device
// allocation, the work lists of the persistent kernels, the step as one CUDA graph, and
// the autotuner of the launch shapes.  The arithmetic is the single-model kernels'
// bodies (ocean_kernels.cu); nothing here touches field values.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ocean.h"
#include "ocean_internal.cuh"

struct ocean_ensemble_s {
    int M = 0, prec = OCEAN_MIXED, ns = 0, npass = 0, nsm = 0;
    std::vector<ocean_t> mem;
    char* arena = nullptr;
    cudaStream_t stream = nullptr;
    // four tables of M entries (index 2 * first + cur), each tab_bytes long
    char* d_tab = nullptr;
    size_t tab_bytes = 0;
    // work items of all kinds back to back; kind k at [off[k], off[k] + cnt[k])
    EnsItem* d_work = nullptr;
    int off[ENS_NKIND] = {}, cnt[ENS_NKIND] = {};
    int* d_counters = nullptr;   // one per launch of a step
    int nlaunch = 0;
    int grid[ENS_NKIND] = {}, dyn[ENS_NKIND] = {}, maxres[ENS_NKIND] = {};
    float tuned_ms[ENS_NKIND] = {};   // best time of each kind's launches in autotuning
    // barotropic regions: the work lists cut for each halo width of ENS_REGION_BS (after
    // the other kinds' in d_work) and the one in use
    int off_bp[3] = {}, cnt_bp[3] = {}, bsi = 1;
    float region_ms[3] = {};          // best sub-cycle pass time of each halo width
    cudaGraphExec_t graph[2] = {};
    long launches = 0;
};

namespace {

int efail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    oc_set_last_error(buf);
    return code;
}

#define EN_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return efail(OCEAN_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Work lists.  Cost estimates only order the items: levels a tile or chunk marches
// through (a tile's deepest wet column), 1 for the 2-D kernels.
void build_work(ocean_ensemble_t e, std::vector<EnsItem> (&w)[ENS_NKIND]) {
    const EnsShape sh = ens_shape();
    for (int m = 0; m < e->M; ++m) {
        const OcMemberInfo I = oc_member_info(e->mem[m]);
        const long ncol = (long)I.nx * I.ny, nring = (long)(I.nx + 2) * (I.ny + 2);
        for (long a = 0; a * sh.chunk < nring; ++a) w[ENS_DIAG].push_back({m, (int)a, 0, I.nz});
        for (long a = 0; a * sh.chunk < ncol; ++a) {
            w[ENS_BARO_BEGIN].push_back({m, (int)a, 0, 1});
            w[ENS_BARO_END].push_back({m, (int)a, 0, 1});
            for (int sl = 0; sl * sh.corr_slab < I.nz; ++sl)
                w[ENS_CORRECT].push_back({m, (int)a, sl, std::min(sh.corr_slab, I.nz - sl * sh.corr_slab)});
        }
        const int ntx = (I.nx + sh.tile_x - 1) / sh.tile_x, nty = (I.ny + sh.tile_y - 1) / sh.tile_y;
        for (int by = 0; by < nty; ++by)
            for (int bx = 0; bx < ntx; ++bx) {
                int kmin = I.nz;
                for (int j = by * sh.tile_y; j < std::min(I.ny, (by + 1) * sh.tile_y); ++j)
                    for (int i = bx * sh.tile_x; i < std::min(I.nx, (bx + 1) * sh.tile_x); ++i)
                        kmin = std::min(kmin, oc_member_kb(e->mem[m], i, j));
                const EnsItem it{m, bx, by, I.nz - kmin};
                w[ENS_TRACER].push_back(it);
                w[ENS_MOMENTUM].push_back(it);
            }
    }
    for (auto& v : w)
        std::stable_sort(v.begin(), v.end(),
                         [](const EnsItem& a, const EnsItem& b) { return a.cost > b.cost; });
}

// the barotropic region items of every member for halo width bs (regions of
// (region_w - 2 bs) x (region_h - 2 bs) interior columns)
std::vector<EnsItem> region_work(ocean_ensemble_t e, int bs) {
    const EnsShape sh = ens_shape();
    const int ix = sh.region_w - 2 * bs, iy = sh.region_h - 2 * bs;
    std::vector<EnsItem> w;
    for (int m = 0; m < e->M; ++m) {
        const OcMemberInfo I = oc_member_info(e->mem[m]);
        const int nrx = (I.nx + ix - 1) / ix, nry = (I.ny + iy - 1) / iy;
        for (int ry = 0; ry < nry; ++ry)
            for (int rx = 0; rx < nrx; ++rx) w.push_back({m, rx, ry, 1});
    }
    return w;
}

// table v (= 2 first + cur) starts at byte v * tab_bytes, where the kernels look for it
template <typename R>
int upload_tables(ocean_ensemble_t e) {
    if (e->tab_bytes < (size_t)e->M * sizeof(EnsMember<R>))
        return efail(OCEAN_ERR_ARG, "ensemble table stride too small");
    std::vector<unsigned char> h(4 * e->tab_bytes, 0);
    for (int first = 0; first < 2; ++first)
        for (int cur = 0; cur < 2; ++cur)
            for (int m = 0; m < e->M; ++m) {
                const EnsMember<R> x = oc_member_entry<R>(e->mem[m], first, cur);
                std::memcpy(h.data() + (size_t)(2 * first + cur) * e->tab_bytes + m * sizeof(x), &x,
                            sizeof(x));
            }
    EN_CUDA(cudaMemcpy(e->d_tab, h.data(), h.size(), cudaMemcpyHostToDevice));
    return OCEAN_OK;
}

template <typename R>
void enqueue_t(ocean_ensemble_t e, int variant, const int* grid, const int* dyn,
               cudaEvent_t* ev) {
    cudaStream_t s = e->stream;
    const EnsMember<R>* tab =
        reinterpret_cast<const EnsMember<R>*>(e->d_tab + (size_t)variant * e->tab_bytes);
    cudaMemsetAsync(e->d_counters, 0, sizeof(int) * e->nlaunch, s);
    int li = 0;
    const int bs = ENS_REGION_BS[e->bsi];
    auto run = [&](int kind, int odd, int nsub) {
        launch_ens<R>(kind, tab, e->d_work + e->off[kind], e->cnt[kind], grid[kind],
                      dyn[kind] ? e->d_counters + li : nullptr, odd, nsub, bs, s);
        ++li;
    };
    auto mark = [&](int k) { if (ev) cudaEventRecord(ev[k], s); };
    mark(0);
    run(ENS_DIAG, 0, 0);
    mark(1);
    run(ENS_TRACER, 0, 0);
    mark(2);
    run(ENS_MOMENTUM, 0, 0);
    mark(3);
    run(ENS_BARO_BEGIN, 0, 0);
    mark(4);
    for (int p = 0, m0 = 0; m0 < e->ns; ++p, m0 += bs)
        run(ENS_BARO_PASS, p & 1, std::min(bs, e->ns - m0));
    mark(5);
    run(ENS_BARO_END, 0, 0);
    mark(6);
    run(ENS_CORRECT, 0, 0);
    mark(7);
}

void enqueue(ocean_ensemble_t e, int variant, const int* grid, const int* dyn, cudaEvent_t* ev) {
    if (e->prec == OCEAN_FP64) enqueue_t<double>(e, variant, grid, dyn, ev);
    else enqueue_t<float>(e, variant, grid, dyn, ev);
}

// the members' common step state: table variant, or -1 if they are out of step
int current_variant(ocean_ensemble_t e) {
    const OcMemberInfo a = oc_member_info(e->mem[0]);
    for (int m = 1; m < e->M; ++m) {
        const OcMemberInfo b = oc_member_info(e->mem[m]);
        if (b.nstep != a.nstep || b.cur != a.cur) return -1;
    }
    return 2 * (a.nstep == 0 ? 1 : 0) + a.cur;
}

void drop_graphs(ocean_ensemble_t e) {
    for (auto& g : e->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

int step_one(ocean_ensemble_t e, const int* grid, const int* dyn, cudaEvent_t* ev) {
    const int v = current_variant(e);
    if (v < 0)
        return efail(OCEAN_ERR_STATE, "ensemble members are out of step (a member was stepped on its own)");
    if (ev || v >= 2) {
        // timed (autotuning) or first (Euler) step: direct launches
        enqueue(e, v, grid, dyn, ev);
    } else {
        if (!e->graph[v]) {
            cudaGraph_t g = nullptr;
            EN_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
            enqueue(e, v, grid, dyn, nullptr);
            EN_CUDA(cudaStreamEndCapture(e->stream, &g));
            cudaError_t r = cudaGraphInstantiate(&e->graph[v], g, 0);
            cudaGraphDestroy(g);
            if (r != cudaSuccess)
                return efail(OCEAN_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(r));
        }
        EN_CUDA(cudaGraphLaunch(e->graph[v], e->stream));
    }
    EN_CUDA(cudaGetLastError());
    for (ocean_t m : e->mem) oc_member_advance(m);
    e->launches += e->nlaunch;
    return OCEAN_OK;
}

void default_shapes(ocean_ensemble_t e) {
    for (int k = 0; k < ENS_NKIND; ++k) {
        e->grid[k] = std::max(1, std::min(e->cnt[k], e->maxres[k] * e->nsm));
        e->dyn[k] = 1;
    }
}

// use the barotropic regions of halo width ENS_REGION_BS[i]: their work list, the number of
// passes of a step, and the default launch shape of the pass kind
void set_region(ocean_ensemble_t e, int i) {
    e->bsi = i;
    e->off[ENS_BARO_PASS] = e->off_bp[i];
    e->cnt[ENS_BARO_PASS] = e->cnt_bp[i];
    e->npass = (e->ns + ENS_REGION_BS[i] - 1) / ENS_REGION_BS[i];
    e->nlaunch = 6 + e->npass;
    const int k = ENS_BARO_PASS;
    e->grid[k] = std::max(1, std::min(e->cnt[k], e->maxres[k] * e->nsm));
    e->dyn[k] = 1;
    drop_graphs(e);
}

}  // namespace

extern "C" {

int ocean_ensemble_create(int members, const ocean_grid* grids, const double* const* depths,
                          const ocean_params* params, ocean_ensemble_t* out) {
    if (!out) return efail(OCEAN_ERR_ARG, "null output handle");
    *out = nullptr;
    if (members < 1 || !grids || !depths || !params)
        return efail(OCEAN_ERR_ARG, "need members >= 1 and non-null grids, depths, params");
    for (int m = 0; m < members; ++m) {
        const ocean_grid& g = grids[m];
        const ocean_params& p = params[m];
        if (g.periodic_x || g.periodic_y)
            return efail(OCEAN_ERR_ARG, "member %d: ensemble members must be closed basins", m);
        if (p.closure != OCEAN_CLOSURE_RI || p.closure_hidden != 0)
            return efail(OCEAN_ERR_ARG, "member %d: ensemble members use the Richardson-number closure", m);
        if (p.vertical_weno != OCEAN_VWENO_INDEX || p.momentum_vadv != OCEAN_VADV_CENTRED)
            return efail(OCEAN_ERR_ARG, "member %d: ensemble members use the default vertical schemes", m);
        if (p.baro_filter != OCEAN_FILTER_BOXCAR)
            return efail(OCEAN_ERR_ARG, "member %d: ensemble members average the sub-cycle with equal weights", m);
        if (p.precision != params[0].precision || p.dt != params[0].dt ||
            p.n_substeps != params[0].n_substeps)
            return efail(OCEAN_ERR_ARG, "member %d: members must share precision, dt and n_substeps", m);
        if (!depths[m]) return efail(OCEAN_ERR_ARG, "member %d: null depth", m);
    }
    ocean_ensemble_t e = new ocean_ensemble_s();
    e->M = members;
    e->prec = params[0].precision;
    e->ns = params[0].n_substeps;
    auto bail = [&](int rc) {
        ocean_ensemble_destroy(e);
        return rc;
    };
    // one allocation for all members
    std::vector<size_t> need(members);
    size_t total = 0;
    for (int m = 0; m < members; ++m) {
        int rc = ocean_arena_bytes(&grids[m], &params[m], &need[m]);
        if (rc) return bail(rc);
        need[m] = align256(need[m]);
        total += need[m];
    }
    cudaError_t ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(efail(OCEAN_ERR_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(ce)));
    ce = cudaMalloc(&e->arena, total);
    if (ce != cudaSuccess) {
        e->arena = nullptr;
        return bail(efail(OCEAN_ERR_OOM, "cudaMalloc of %zu bytes for the ensemble failed: %s", total, cudaGetErrorString(ce)));
    }
    size_t at = 0;
    for (int m = 0; m < members; ++m) {
        ocean_t h = nullptr;
        int rc = oc_member_create(&grids[m], depths[m], &params[m], e->arena + at, need[m],
                                  e->stream, &h);
        if (rc) return bail(rc);
        e->mem.push_back(h);
        at += need[m];
    }
    // work lists and tables
    std::vector<EnsItem> w[ENS_NKIND];
    build_work(e, w);
    std::vector<EnsItem> all;
    for (int k = 0; k < ENS_NKIND; ++k) {
        e->off[k] = (int)all.size();
        e->cnt[k] = (int)w[k].size();
        all.insert(all.end(), w[k].begin(), w[k].end());
    }
    int max_launch = 0;
    for (int i = 0; i < 3; ++i) {
        const std::vector<EnsItem> r = region_work(e, ENS_REGION_BS[i]);
        e->off_bp[i] = (int)all.size();
        e->cnt_bp[i] = (int)r.size();
        all.insert(all.end(), r.begin(), r.end());
        max_launch = std::max(max_launch, 6 + (e->ns + ENS_REGION_BS[i] - 1) / ENS_REGION_BS[i]);
        if (ENS_REGION_BS[i] == ens_shape().pass_substeps) e->bsi = i;
    }
    e->tab_bytes = align256(members * (e->prec == OCEAN_FP64 ? sizeof(EnsMember<double>)
                                                            : sizeof(EnsMember<float>)));
    if ((ce = cudaMalloc(&e->d_tab, 4 * e->tab_bytes)) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_work, all.size() * sizeof(EnsItem))) != cudaSuccess ||
        (ce = cudaMalloc(&e->d_counters, sizeof(int) * max_launch)) != cudaSuccess)
        return bail(efail(OCEAN_ERR_OOM, "ensemble tables: %s", cudaGetErrorString(ce)));
    ce = cudaMemcpy(e->d_work, all.data(), all.size() * sizeof(EnsItem), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bail(efail(OCEAN_ERR_CUDA, "work list upload: %s", cudaGetErrorString(ce)));
    int rc = e->prec == OCEAN_FP64 ? upload_tables<double>(e) : upload_tables<float>(e);
    if (rc) return bail(rc);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < ENS_NKIND; ++k) {
        e->maxres[k] = e->prec == OCEAN_FP64 ? ens_blocks_per_sm<double>(k) : ens_blocks_per_sm<float>(k);
        if (e->maxres[k] < 1) return bail(efail(OCEAN_ERR_CUDA, "ensemble kernel %d cannot be resident", k));
    }
    set_region(e, e->bsi);
    default_shapes(e);
    *out = e;
    return OCEAN_OK;
}

void ocean_ensemble_destroy(ocean_ensemble_t e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    drop_graphs(e);
    for (ocean_t m : e->mem) ocean_destroy(m);
    cudaFree(e->d_tab);
    cudaFree(e->d_work);
    cudaFree(e->d_counters);
    cudaFree(e->arena);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

int ocean_ensemble_size(ocean_ensemble_t e) { return e ? e->M : 0; }

ocean_t ocean_ensemble_member(ocean_ensemble_t e, int i) {
    return (e && i >= 0 && i < e->M) ? e->mem[i] : nullptr;
}

void* ocean_ensemble_stream(ocean_ensemble_t e) { return e ? (void*)e->stream : nullptr; }

int ocean_ensemble_step_async(ocean_ensemble_t e, int n) {
    if (!e) return efail(OCEAN_ERR_ARG, "null ensemble");
    if (n < 0) return efail(OCEAN_ERR_ARG, "negative step count");
    for (int i = 0; i < n; ++i) {
        int rc = step_one(e, e->grid, e->dyn, nullptr);
        if (rc) return rc;
    }
    return OCEAN_OK;
}

int ocean_ensemble_step(ocean_ensemble_t e, int n) {
    int rc = ocean_ensemble_step_async(e, n);
    if (rc) return rc;
    EN_CUDA(cudaStreamSynchronize(e->stream));
    if (tile_wait_failed())
        return efail(OCEAN_ERR_TIMEOUT, "a tile kernel's wait for its tensor copies timed out");
    return OCEAN_OK;
}

int ocean_ensemble_autotune(ocean_ensemble_t e, int reps, int* steps_taken) {
    if (!e) return efail(OCEAN_ERR_ARG, "null ensemble");
    if (reps < 1) return efail(OCEAN_ERR_ARG, "reps must be >= 1");
    if (steps_taken) *steps_taken = 0;
    // candidates per kind: one item per block, then persistent grids x schedules
    struct Cand { int grid, dyn; };
    std::vector<Cand> cand[ENS_NKIND];
    size_t ncmax = 1;
    for (int k = 0; k < ENS_NKIND; ++k) {
        const int W = std::max(1, e->cnt[k]);
        cand[k].push_back({W, 0});
        std::vector<int> grids = {e->nsm, 2 * e->nsm, e->maxres[k] * e->nsm};
        std::sort(grids.begin(), grids.end());
        grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
        for (int g : grids) {
            if (g >= W) continue;
            cand[k].push_back({g, 0});
            cand[k].push_back({g, 1});
        }
        ncmax = std::max(ncmax, cand[k].size());
    }
    cudaEvent_t ev[8];
    for (auto& x : ev) cudaEventCreate(&x);
    std::vector<std::vector<float>> ms(ENS_NKIND);
    for (int k = 0; k < ENS_NKIND; ++k) ms[k].assign(cand[k].size(), 3.4e38f);
    const int kind_at[7] = {ENS_DIAG, ENS_TRACER, ENS_MOMENTUM, ENS_BARO_BEGIN, ENS_BARO_PASS,
                            ENS_BARO_END, ENS_CORRECT};
    int rc = OCEAN_OK, taken = 0;
    for (int r = 0; r < reps && rc == OCEAN_OK; ++r)
        for (size_t t = 0; t < ncmax && rc == OCEAN_OK; ++t) {
            int grid[ENS_NKIND], dyn[ENS_NKIND];
            for (int k = 0; k < ENS_NKIND; ++k) {
                const Cand& c = cand[k][t % cand[k].size()];
                grid[k] = c.grid;
                dyn[k] = c.dyn;
            }
            rc = step_one(e, grid, dyn, ev);
            if (rc) break;
            ++taken;
            if (cudaEventSynchronize(ev[7]) != cudaSuccess) {
                rc = efail(OCEAN_ERR_CUDA, "autotune step failed: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            for (int q = 0; q < 7; ++q) {
                float x = 0.f;
                cudaEventElapsedTime(&x, ev[q], ev[q + 1]);
                const int k = kind_at[q];
                float& best = ms[k][t % cand[k].size()];
                best = std::min(best, x);
            }
        }
    for (auto& x : ev) cudaEventDestroy(x);
    if (steps_taken) *steps_taken = taken;
    if (rc) return rc;
    for (int k = 0; k < ENS_NKIND; ++k) {
        size_t b = 0;
        for (size_t c = 1; c < cand[k].size(); ++c)
            if (ms[k][c] < ms[k][b]) b = c;
        e->grid[k] = cand[k][b].grid;
        e->dyn[k] = cand[k][b].dyn;
        e->tuned_ms[k] = ms[k][b];
    }
    drop_graphs(e);
    return OCEAN_OK;
}

int ocean_ensemble_autotune_regions(ocean_ensemble_t e, int reps, int* steps_taken) {
    if (!e) return efail(OCEAN_ERR_ARG, "null ensemble");
    if (reps < 1) return efail(OCEAN_ERR_ARG, "reps must be >= 1");
    if (steps_taken) *steps_taken = 0;
    cudaEvent_t ev[8];
    for (auto& x : ev) cudaEventCreate(&x);
    int rc = OCEAN_OK, taken = 0;
    for (int i = 0; i < 3 && rc == OCEAN_OK; ++i) {
        if (ENS_REGION_BS[i] > e->ns && i != e->bsi) {   // a wider halo than the sub-cycle
            e->region_ms[i] = 3.4e38f;
            continue;
        }
        set_region(e, i);
        float ms = 3.4e38f;
        for (int r = 0; r < reps && rc == OCEAN_OK; ++r) {
            rc = step_one(e, e->grid, e->dyn, ev);
            if (rc) break;
            ++taken;
            if (cudaEventSynchronize(ev[7]) != cudaSuccess) {
                rc = efail(OCEAN_ERR_CUDA, "region autotune step failed: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float x = 0.f;
            cudaEventElapsedTime(&x, ev[4], ev[5]);   // the sub-cycle's passes
            ms = std::min(ms, x);
        }
        e->region_ms[i] = ms;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (steps_taken) *steps_taken = taken;
    if (rc) return rc;
    int b = 0;
    for (int i = 1; i < 3; ++i)
        if (e->region_ms[i] < e->region_ms[b]) b = i;
    set_region(e, b);
    return OCEAN_OK;
}

int ocean_ensemble_region_substeps(ocean_ensemble_t e) { return e ? ENS_REGION_BS[e->bsi] : 0; }

int ocean_ensemble_set_region_substeps(ocean_ensemble_t e, int bs) {
    if (!e) return efail(OCEAN_ERR_ARG, "null ensemble");
    for (int i = 0; i < 3; ++i)
        if (ENS_REGION_BS[i] == bs) {
            set_region(e, i);
            return OCEAN_OK;
        }
    return efail(OCEAN_ERR_ARG, "region substeps %d: choose 4, 6 or 8", bs);
}

int ocean_ensemble_region_times(ocean_ensemble_t e, float* ms) {
    if (!e || !ms) return efail(OCEAN_ERR_ARG, "null argument");
    for (int i = 0; i < 3; ++i) ms[i] = e->region_ms[i];
    return OCEAN_OK;
}

int ocean_ensemble_launch_shapes(ocean_ensemble_t e, int* grid, int* dynamic, int* items) {
    if (!e) return efail(OCEAN_ERR_ARG, "null ensemble");
    for (int k = 0; k < ENS_NKIND; ++k) {
        if (grid) grid[k] = e->grid[k];
        if (dynamic) dynamic[k] = e->dyn[k];
        if (items) items[k] = e->cnt[k];
    }
    return OCEAN_OK;
}

long ocean_ensemble_kernel_launches(ocean_ensemble_t e) { return e ? e->launches : -1; }

int ocean_ensemble_kind_times(ocean_ensemble_t e, double* ms) {
    if (!e || !ms) return efail(OCEAN_ERR_ARG, "null ensemble or output");
    for (int k = 0; k < ENS_NKIND; ++k) ms[k] = e->tuned_ms[k];
    return OCEAN_OK;
}

}  // extern "C"
