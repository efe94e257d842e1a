// C-ABI entry points (include/ep.h): contexts, jobs, batched stepping with
// CUDA-graph replay, state transfer. Host-side runtime only; every step of
// the method runs in the kernels of kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <set>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ep.h"
#include "devtypes.h"
#include "graph_plan.h"
#include "bidomain.h"
#include "kernels.h"
#include "planner.h"
#include "varmap.h"

using namespace ep;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

constexpr int kGraphSteps = 32;       // steps per captured graph
constexpr size_t kMaxPlans = 512;     // cached batch plans per context (job tables, tiles, graphs)
constexpr int kGraphMinSteps = 64;    // below this, launch directly

struct Plan {
    std::vector<ep_job *> jobs;
    std::vector<uint64_t> versions;
    struct Group {
        int precision;
        int n_jobs;
        DevBuf jobtab, node_tiles, cell_tiles, done, graph_tiles, graph_sub_tiles, work;
        StepLaunch L;
        // host copies of the descriptors of a group of one job (L.tab1) or of at most kParamJobs
        // jobs (L.tabk), passed to the FP32 kernels as a parameter
        std::shared_ptr<JobTab<1>> tab1;
        std::shared_ptr<JobTab<kParamJobs>> tabk;
    };
    std::vector<Group> groups;
    std::vector<ep_job *> bido;   // jobs whose step ends with the elliptic solve
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

// Bidomain state of a job (ep_bidomain_enable).
struct BidoHost {
    std::vector<double> De_l, De_t;   // extracellular diffusivities per parameter set
    double tol = 1e-6, atol = 0.0;
    double barrier_limit_s = 2.0;
    int restart = 12;
    int reorth = 0;
    int64_t max_iter = 2000;
    std::vector<DevBuf> bufs;
    BidoArgs args{};
    int grid = 1;
};

}  // namespace

struct ep_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    cudaStream_t upload = nullptr;   // job creation uploads: never waits on queued steps
    ep_alloc_fn alloc = nullptr;
    ep_free_fn free_fn = nullptr;
    void *user = nullptr;
    std::string err;
    std::set<ep_job *> jobs;
    std::vector<std::unique_ptr<Plan>> plans;
    int sm_count = 148;
    int cell_variant[2] = {0, 0};   // launch shape of the cell kernel per precision (ep_autotune)
    int graph_mode = EP_GRAPH_SUBSTEPS_LOCAL;   // ep_set_graph_kernel
    DevBuf err_word;                 // device word: a bounded wait in a step kernel gave up
    unsigned *err_host = nullptr;    // pinned copy of err_word, refreshed after each ep_step of staged kernels
};

struct ep_job {
    ep_context *ctx = nullptr;
    std::shared_ptr<HostMesh> mp;   // shared with the ep_plan it came from, if any
    std::shared_ptr<Sell> sp;
    const HostMesh &mesh() const { return *mp; }
    const Sell &sell() const { return *sp; }
    bool has_params = false;
    ep_params params{};
    int precision = -1;
    uint64_t version = 1;
    DevJob dj{};
    DevBuf dj_dev;
    DevBuf step_dev;
    const int *perm_dev = nullptr;  // internal cell -> caller cell
    std::vector<DevBuf> topo;     // precision-independent device arrays
    std::vector<DevBuf> prec;     // precision-dependent device arrays
    std::vector<Tile> cell_tiles, node_tiles;
    std::vector<int2> cell_deps;  // per cell tile: the node tiles (node >> 8) its gathers read, [x, y]
    int64_t device_bytes = 0;
    // conduction graph (ep_graph_attach)
    std::unique_ptr<GraphPlan> gp;
    std::vector<DevBuf> gbufs;
    std::vector<Tile> graph_tiles;
    int graph_lmax = 0;              // largest local slot count of the graph's tiles (one-launch substeps)
    const int *gperm_dev = nullptr;
    DevBuf graph_view;               // DevJob whose V/act/regions are the graph's (init, I/O)
    // bidomain (ep_bidomain_enable)
    std::unique_ptr<BidoHost> bido;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(ep_context *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(ep_context *ctx, cudaError_t e, const char *what) {
    return fail(ctx, EP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int dalloc(ep_context *ctx, size_t bytes, DevBuf *b) {
    bytes = std::max<size_t>(bytes, 256);
    void *p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(bytes, ctx->user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) return fail(ctx, EP_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    b->p = p;
    b->bytes = bytes;
    return EP_OK;
}

void dfree(ep_context *ctx, DevBuf *b) {
    if (!b->p) return;
    if (ctx->free_fn) ctx->free_fn(b->p, b->bytes, ctx->user);
    else cudaFree(b->p);
    b->p = nullptr;
    b->bytes = 0;
}

template <class T>
int upload(ep_context *ctx, const std::vector<T> &v, std::vector<DevBuf> *pool, void **out) {
    DevBuf b;
    int rc = dalloc(ctx, v.size() * sizeof(T), &b);
    if (rc) return rc;
    pool->push_back(b);
    if (!v.empty()) {
        cudaError_t e = cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->upload);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
        e = cudaStreamSynchronize(ctx->upload);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
    }
    *out = b.p;
    return EP_OK;
}

void free_plan(ep_context *ctx, Plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &g : p->groups) {
        dfree(ctx, &g.jobtab);
        dfree(ctx, &g.node_tiles);
        dfree(ctx, &g.cell_tiles);
        dfree(ctx, &g.done);
        dfree(ctx, &g.graph_tiles);
        dfree(ctx, &g.graph_sub_tiles);
        dfree(ctx, &g.work);
    }
}

void drop_plans_with(ep_context *ctx, ep_job *job) {
    auto &pl = ctx->plans;
    for (size_t i = 0; i < pl.size();) {
        if (std::find(pl[i]->jobs.begin(), pl[i]->jobs.end(), job) != pl[i]->jobs.end()) {
            free_plan(ctx, pl[i].get());
            pl.erase(pl.begin() + i);
        } else {
            ++i;
        }
    }
}

void free_job_arrays(ep_job *j, std::vector<DevBuf> *pool) {
    for (auto &b : *pool) dfree(j->ctx, &b);
    pool->clear();
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Tiles of at most kCellThreads consecutive cells inside one model region,
// kNodeThreads consecutive nodes (starting on a 32-node slice).
void build_tiles(ep_job *j) {
    j->cell_tiles.clear();
    j->node_tiles.clear();
    for (int m = 0; m < EP_N_MODELS; ++m)
        for (int64_t s = j->mesh().model_off[m]; s < j->mesh().model_off[m + 1]; s += kCellThreads)
            j->cell_tiles.push_back(Tile{0, m, int(s), int(std::min<int64_t>(kCellThreads, j->mesh().model_off[m + 1] - s))});
    for (int64_t s = 0; s < j->mesh().n_nodes; s += kNodeThreads)
        j->node_tiles.push_back(Tile{0, 0, int(s), int(std::min<int64_t>(kNodeThreads, j->mesh().n_nodes - s))});
    j->cell_deps.clear();
    for (const Tile &t : j->cell_tiles) {
        int32_t lo = INT32_MAX, hi = 0, na[4], nb[4], nc[4];
        for (int64_t c = t.start; c < t.start + t.count; ++c) {
            cell_gather_indices(j->mesh(), c, na, nb, nc);
            for (int k = 0; k < 4; ++k) lo = std::min({lo, na[k], nb[k]}), hi = std::max({hi, na[k], nb[k]});
        }
        j->cell_deps.push_back(make_int2(lo / kNodeThreads, hi / kNodeThreads));
    }
}

// Work list of the fused step for one job whose tiles sit at node_off / cell_off
// in the launch's tile tables: every cell tile is preceded by the node tiles its
// gathers read -- node tiles are queued in increasing order up to the largest
// one needed by the next kFusedLookahead cell tiles -- so a cell tile only ever
// waits for node tiles claimed before it.
void append_work(const ep_job *j, int node_off, int cell_off, std::vector<Work> *w) {
    const int nct = int(j->cell_tiles.size()), nnt = int(j->node_tiles.size());
    std::vector<int> pmax(nct);
    for (int t = 0; t < nct; ++t) pmax[t] = std::max(t ? pmax[t - 1] : 0, j->cell_deps[t].y);
    int next = 0;
    for (int t = 0; t < nct; ++t) {
        const int need = pmax[std::min(nct - 1, t + kFusedLookahead)];
        for (; next <= need && next < nnt; ++next) w->push_back(Work{-1 - (node_off + next), 0, 0, 0});
        w->push_back(Work{cell_off + t, j->cell_deps[t].x, j->cell_deps[t].y, 0});
    }
    for (; next < nnt; ++next) w->push_back(Work{-1 - (node_off + next), 0, 0, 0});
}

}  // namespace

extern "C" {

int ep_context_create(ep_alloc_fn alloc, ep_free_fn free_fn, void *user, void *cuda_stream, ep_context **out) {
    if (!out || (alloc == nullptr) != (free_fn == nullptr)) {
        g_create_error = "ep_context_create: out is NULL or only one of alloc/free given";
        return EP_EINVAL;
    }
    try {
        auto *ctx = new ep_context();
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->upload, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("ep_context_create: ") + cudaGetErrorString(e);
            delete ctx;
            return EP_ECUDA;
        }
        ctx->alloc = alloc;
        ctx->free_fn = free_fn;
        ctx->user = user;
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
        // the error word is the context's own (cudaMalloc), outside the caller's allocator budget
        if (cudaMalloc(&ctx->err_word.p, sizeof(unsigned)) != cudaSuccess ||
            cudaMemset(ctx->err_word.p, 0, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            g_create_error = "ep_context_create: device allocation failed";
            if (ctx->err_word.p) cudaFree(ctx->err_word.p);
            cudaStreamDestroy(ctx->capture);
            cudaStreamDestroy(ctx->upload);
            delete ctx;
            return EP_ENOMEM;
        }
        if (cudaHostAlloc(reinterpret_cast<void **>(&ctx->err_host), sizeof(unsigned), cudaHostAllocDefault) !=
            cudaSuccess) {
            cudaGetLastError();
            g_create_error = "ep_context_create: pinned host allocation failed";
            cudaFree(ctx->err_word.p);
            cudaStreamDestroy(ctx->capture);
            cudaStreamDestroy(ctx->upload);
            delete ctx;
            return EP_ENOMEM;
        }
        *ctx->err_host = 0u;
        *out = ctx;
        return EP_OK;
    } catch (...) {
        g_create_error = "ep_context_create: out of host memory";
        return EP_ENOMEM;
    }
}

int ep_context_set_stream(ep_context *ctx, void *cuda_stream) {
    if (!ctx) return EP_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return EP_OK;
}

int ep_context_destroy(ep_context *ctx) {
    if (!ctx) return EP_EINVAL;
    if (!ctx->jobs.empty()) return fail(ctx, EP_ESTATE, "ep_context_destroy: jobs still alive");
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &p : ctx->plans) free_plan(ctx, p.get());
    ctx->plans.clear();
    if (ctx->err_word.p) cudaFree(ctx->err_word.p);
    if (ctx->err_host) cudaFreeHost(ctx->err_host);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    if (ctx->upload) cudaStreamDestroy(ctx->upload);
    delete ctx;
    return EP_OK;
}

int ep_set_graph_kernel(ep_context *ctx, int32_t mode) {
    if (!ctx) return EP_EINVAL;
    if (mode != EP_GRAPH_SUBSTEPS_LAUNCHES && mode != EP_GRAPH_SUBSTEPS_LOCAL)
        return fail(ctx, EP_EINVAL, "ep_set_graph_kernel: unknown mode");
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->graph_mode = mode;
    for (auto &p : ctx->plans) free_plan(ctx, p.get());   // rebuilt with the new mode on next use
    ctx->plans.clear();
    return EP_OK;
}

int ep_clear_error(ep_context *ctx) {
    if (!ctx) return EP_EINVAL;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->err_word.p, 0, sizeof(unsigned), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_clear_error");
    *ctx->err_host = 0u;
    return EP_OK;
}

const char *ep_last_error(const ep_context *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int32_t ep_model_nvar(int32_t model) { return model_nvar(model); }

const char *ep_model_varname(int32_t model, int32_t var) {
    if (var < 0 || var >= model_nvar(model)) return nullptr;
    return model_vars(model)[var].name;
}

int32_t ep_model_var_compensated(int32_t model, int32_t var) {
    if (model < 0 || model >= EP_N_MODELS || var < 0 || var >= model_nvar(model)) return -1;
    return model_vars(model)[var].kind == kVarA ? 1 : 0;
}

int64_t ep_estimate_bytes(int64_t n_cells, int64_t n_nodes, int32_t precision) {
    const int64_t r = precision == EP_FP64_PLAIN ? 8 : 4;
    // topology: nodes_a/b, nbr (3 int4), pset, smask, sell columns (~4.3 per cell)
    int64_t b = n_cells * (48 + 2) + int64_t(4.4 * n_cells) * 4;
    // coefficients (3 x vec4), V x2, act, sell weights, node values
    b += n_cells * (12 * r + 3 * r) + int64_t(4.4 * n_cells) * r + n_nodes * r;
    // state: up to 16 compute-type + 4 FP64 variables
    b += n_cells * (16 * r + 4 * 8);
    return b + (1 << 20);
}

}  // extern "C"

namespace {

int graph_apply(ep_job *job);
int bido_apply(ep_job *job);
void bido_drop(ep_job *job);
int restart_ab2(ep_job *job);

// Validate a parameter block and fold it into FP64 coefficients for a mesh,
// with the explicit stability check dt * rho(L) < 2 (host only).
int plan_params(const HostMesh &m, const ep_params *p, Coeffs *cf, std::string *err) {
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) {
        *err = "params: dt must be > 0";
        return EP_EINVAL;
    }
    if (p->precision != EP_FP32_MIXED && p->precision != EP_FP64_PLAIN) {
        *err = "params: unknown precision";
        return EP_EINVAL;
    }
    if (p->n_sets < 1 || p->n_sets > EP_MAX_PARAM_SETS || p->n_stim < 0 || p->n_stim > EP_MAX_STIMULI) {
        *err = "params: n_sets must be 1..16 and n_stim 0..8";
        return EP_EINVAL;
    }
    if (p->integrator != EP_INTEGRATOR_FE && p->integrator != EP_INTEGRATOR_AB2) {
        *err = "params: unknown integrator";
        return EP_EINVAL;
    }
    for (int s = 0; s < p->n_sets; ++s) {
        const ep_cell_params &c = p->sets[s];
        if (!(c.D_l >= 0.0) || !(c.D_t >= 0.0) || !(c.K_o > 0.0) || c.variant < 0 || c.variant > 2) {
            *err = "params: bad parameter set " + std::to_string(s);
            return EP_EINVAL;
        }
    }
    int rc = build_coeffs(m, p, cf, err);
    if (rc) return rc;
    // explicit stability on the diffusion operator's spectrum (real, in [-rho, 0]):
    // forward Euler needs dt rho < 2, AB2 (stability interval [-1, 0]) dt rho < 1
    const double lim = p->integrator == EP_INTEGRATOR_AB2 ? 1.0 : 2.0;
    double rho = cf->gershgorin;
    if (p->dt * rho >= 0.95 * lim) rho = 1.05 * power_radius(m, *cf, 60);
    if (p->dt * rho >= lim) {
        *err = "params: dt = " + std::to_string(p->dt) + " ms exceeds the explicit stability bound " +
               std::to_string(lim / rho) + " ms of the diffusion operator" +
               (p->integrator == EP_INTEGRATOR_AB2 ? " under AB2" : "");
        return EP_EUNSTABLE;
    }
    return EP_OK;
}

// Upload a job's precision-independent arrays (on the context's upload stream).
int job_upload_topology(ep_context *ctx, ep_job *j) {
    const HostMesh &m = j->mesh();
    const Sell &sl = j->sell();
    const int64_t N = m.n_cells;
    void *p;
    int rc;
    j->dj.idx16 = sl.idx16 ? 1 : 0;
    j->dj.col16 = sl.col16ok ? 1 : 0;
    if (sl.col16ok) {
        if ((rc = upload(ctx, sl.col16, &j->topo, &p))) return rc;
        j->dj.ncol16 = static_cast<const unsigned short *>(p);
        if ((rc = upload(ctx, sl.cbase, &j->topo, &p))) return rc;
        j->dj.cbase = static_cast<const int *>(p);
    } else {
        if ((rc = upload(ctx, sl.col, &j->topo, &p))) return rc;
        j->dj.ncol = static_cast<const int *>(p);
    }
    if (sl.idx16) {
        // 16-bit gather indices (offsets; see Sell)
        if ((rc = upload(ctx, sl.cidx16, &j->topo, &p))) return rc;
        j->dj.cidx16 = static_cast<const uint4 *>(p);
        if ((rc = upload(ctx, sl.nbr16, &j->topo, &p))) return rc;
        j->dj.nbr16 = static_cast<const uint2 *>(p);
        if ((rc = upload(ctx, sl.nbase, &j->topo, &p))) return rc;
        j->dj.nbase = static_cast<const int *>(p);
    } else {
        std::vector<int4> na(N), nb(N), nc(N);
        for (int64_t c = 0; c < N; ++c) {
            int32_t a[4], b[4], q[4];
            cell_gather_indices(m, c, a, b, q);
            na[c] = make_int4(a[0], a[1], a[2], a[3]);
            nb[c] = make_int4(b[0], b[1], b[2], b[3]);
            nc[c] = make_int4(q[0], q[1], q[2], q[3]);
        }
        if ((rc = upload(ctx, na, &j->topo, &p))) return rc;
        j->dj.nodes_a = static_cast<const int4 *>(p);
        if ((rc = upload(ctx, nb, &j->topo, &p))) return rc;
        j->dj.nodes_b = static_cast<const int4 *>(p);
        if ((rc = upload(ctx, nc, &j->topo, &p))) return rc;
        j->dj.nbr = static_cast<const int4 *>(p);
    }
    if ((rc = upload(ctx, m.pset, &j->topo, &p))) return rc;
    j->dj.pset = static_cast<const uint8_t *>(p);
    if ((rc = upload(ctx, m.smask, &j->topo, &p))) return rc;
    j->dj.smask = static_cast<const uint8_t *>(p);
    std::vector<long long> sp(sl.slice_ptr.begin(), sl.slice_ptr.end());
    if ((rc = upload(ctx, sp, &j->topo, &p))) return rc;
    j->dj.slice_ptr = static_cast<const long long *>(p);
    if ((rc = upload(ctx, m.cell_new2old, &j->topo, &p))) return rc;
    j->perm_dev = static_cast<const int *>(p);
    DevBuf b;
    // the step counter, and beside it the fused launches' counter (tags of the node-tile flags)
    if ((rc = dalloc(ctx, 2 * sizeof(long long), &b))) return rc;
    j->step_dev = b;
    cudaError_t e = cudaMemsetAsync(b.p, 0, 2 * sizeof(long long), ctx->upload);
    j->dj.step = static_cast<long long *>(b.p);
    j->dj.gen = reinterpret_cast<unsigned *>(static_cast<long long *>(b.p) + 1);
    const int64_t n_chunks = ((m.n_nodes + kNodeThreads - 1) / kNodeThreads + kFusedChunk - 1) / kFusedChunk;
    if ((rc = dalloc(ctx, size_t(n_chunks) * sizeof(unsigned), &b))) return rc;
    j->topo.push_back(b);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.p, 0, size_t(n_chunks) * sizeof(unsigned), ctx->upload);
    j->dj.ntflag = static_cast<unsigned *>(b.p);
    if ((rc = dalloc(ctx, sizeof(DevJob), &b))) return rc;
    j->dj_dev = b;
    j->dj.n_cells = N;
    j->dj.n_nodes = m.n_nodes;
    build_tiles(j);
    for (auto &t : j->topo) j->device_bytes += t.bytes;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "job topology upload");
}

// Upload coefficients and parameters; on the first call (or a precision
// change) allocate the state and set it to the models' resting states.
int job_apply_params(ep_job *job, const ep_params *p, const Coeffs &cf) {
    ep_context *ctx = job->ctx;
    const bool fresh = !job->has_params || job->precision != p->precision ||
                       job->params.integrator != p->integrator;
    if (job->has_params) {
        cudaStreamSynchronize(ctx->stream);
        drop_plans_with(ctx, job);
    }
    const HostMesh &m = job->mesh();
    const Sell &sl = job->sell();
    const int64_t N = m.n_cells;
    std::vector<DevBuf> newprec;
    DevJob dj = job->dj;
    int rc;
    auto put = [&](auto &vec, void **dst) { return upload(ctx, vec, &newprec, dst); };
    auto coeff_upload = [&](const std::vector<double> &v, const void **dst) -> int {
        void *q = nullptr;
        int r;
        if (p->precision == EP_FP64_PLAIN) {
            r = put(v, &q);
        } else {
            std::vector<float> f(v.begin(), v.end());
            r = put(f, &q);
        }
        *dst = q;
        return r;
    };
    std::vector<double> nwd(sl.col.size());
    for (size_t k = 0; k < nwd.size(); ++k) nwd[k] = sl.src[k] >= 0 ? cf.nw[sl.src[k]] : 0.0;
    if ((rc = coeff_upload(cf.wa, &dj.wa)) || (rc = coeff_upload(cf.wb, &dj.wb)) || (rc = coeff_upload(cf.q, &dj.q)) ||
        (rc = coeff_upload(nwd, &dj.nw))) {
        for (auto &b : newprec) dfree(ctx, &b);
        return rc;
    }
    if (fresh) {
        const size_t r = p->precision == EP_FP64_PLAIN ? 8 : 4;
        DevBuf b;
        auto grab = [&](size_t bytes, void **dst) {
            int r2 = dalloc(ctx, bytes, &b);
            if (!r2) {
                newprec.push_back(b);
                *dst = b.p;
            }
            return r2;
        };
        rc = grab(N * r, &dj.V[0]);
        if (!rc) rc = grab(N * r, &dj.V[1]);
        if (!rc) rc = grab(N * r, &dj.act);
        if (!rc) rc = grab(m.n_nodes * r, &dj.vn);
        for (int md = 0; md < EP_N_MODELS && !rc; ++md) {
            DevRegion &rg = dj.reg[md];
            rg.off = m.model_off[md];
            rg.n = m.model_off[md + 1] - m.model_off[md];
            rg.stride = round_up(std::max<int64_t>(rg.n, 1), 64);
            rg.r = nullptr;
            rg.a = nullptr;
            if (rg.n == 0) continue;
            void *q = nullptr;
            rc = grab(size_t(model_nr(md)) * rg.stride * r, &rg.r);
            if (!rc) rc = grab(size_t(model_na(md)) * rg.stride * 8, &q);
            rg.a = static_cast<double *>(q);
            rg.h = nullptr;
            if (!rc && p->integrator == EP_INTEGRATOR_AB2) rc = grab(size_t(kHistSlots) * rg.stride * r, &rg.h);
        }
        if (rc) {
            for (auto &bb : newprec) dfree(ctx, &bb);
            return rc;
        }
    }
    for (int s = 0; s < EP_MAX_PARAM_SETS; ++s) {
        const ep_cell_params &c = p->sets[s < p->n_sets ? s : 0];
        const double sq = std::sqrt(c.K_o / 5.4);
        dj.params[s] = DevParams{c.variant, 0, c.gks_scale, c.gkr_scale, c.K_o, sq,
                                 float(c.gks_scale), float(c.gkr_scale), float(c.K_o), float(sq)};
    }
    dj.n_stim = p->n_stim;
    for (int k = 0; k < p->n_stim; ++k) {
        const ep_stimulus &s = p->stim[k];
        dj.stim[k] = DevStim{s.amplitude, std::llround(s.t_on / p->dt), std::llround(s.duration / p->dt),
                             std::llround(s.period / p->dt), float(s.amplitude), 0};
    }
    dj.precision = p->precision;
    dj.integrator = p->integrator;
    dj.ab2_from = 0;
    if (!fresh && p->integrator == EP_INTEGRATOR_AB2) {   // the AB2 history restarts at the current step
        long long cur = 0;
        if (cudaMemcpy(&cur, job->step_dev.p, sizeof(cur), cudaMemcpyDeviceToHost) == cudaSuccess) dj.ab2_from = cur;
    }
    dj.dt = p->dt;
    dj.threshold = p->threshold;
    dj.dt_f = float(p->dt);
    dj.threshold_f = float(p->threshold);
    // coefficient arrays are always new (the first 4 entries of prec); state arrays only when fresh
    if (fresh) {
        free_job_arrays(job, &job->prec);
        job->prec = newprec;
    } else {
        for (int k = 0; k < 4; ++k) dfree(ctx, &job->prec[k]);
        for (int k = 0; k < 4; ++k) job->prec[k] = newprec[k];
    }
    job->dj = dj;
    cudaError_t e = cudaMemcpyAsync(job->dj_dev.p, &job->dj, sizeof(DevJob), cudaMemcpyHostToDevice, ctx->upload);
    if (e == cudaSuccess && fresh) {
        e = cudaMemsetAsync(job->step_dev.p, 0, sizeof(long long), ctx->upload);
        if (e == cudaSuccess) e = launch_init(p->precision, static_cast<const DevJob *>(job->dj_dev.p), N, ctx->upload);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "params upload");
    job->params = *p;
    job->precision = p->precision;
    job->has_params = true;
    job->version++;
    job->device_bytes = 0;
    for (auto &t : job->topo) job->device_bytes += t.bytes;
    for (auto &t : job->prec) job->device_bytes += t.bytes;
    if (job->gp && (rc = graph_apply(job))) return rc;
    if (job->bido && (rc = bido_apply(job))) {
        bido_drop(job);
        return rc;
    }
    return EP_OK;
}

// Device bytes a job built from this mesh holds once parameters of the given
// precision are set (the allocations of job_upload_topology + job_apply_params).
int64_t job_bytes(const HostMesh &m, const Sell &sl, int precision, int integrator = EP_INTEGRATOR_FE) {
    auto rnd = [](int64_t b) { return std::max<int64_t>(b, 256); };
    const int64_t N = m.n_cells, r = precision == EP_FP64_PLAIN ? 8 : 4, E = int64_t(sl.col.size());
    const int64_t ns = int64_t(sl.slice_ptr.size()) - 1;
    int64_t b = 2 * rnd(N) + rnd(8 * int64_t(sl.slice_ptr.size())) + rnd(4 * N) + 256 + rnd(sizeof(DevJob)) +
                rnd(4 * (((m.n_nodes + kNodeThreads - 1) / kNodeThreads + kFusedChunk - 1) / kFusedChunk));
    b += sl.idx16 ? rnd(16 * N) + rnd(8 * N) + rnd(4 * ((N + 255) / 256)) : 3 * rnd(16 * N);
    b += sl.col16ok ? rnd(2 * E) + rnd(4 * ns) : rnd(4 * E);
    b += 3 * rnd(4 * r * N) + rnd(r * E) + 3 * rnd(r * N) + rnd(r * m.n_nodes);
    for (int md = 0; md < EP_N_MODELS; ++md) {
        const int64_t n = m.model_off[md + 1] - m.model_off[md];
        if (!n) continue;
        const int64_t stride = round_up(n, 64);
        b += rnd(model_nr(md) * stride * r) + rnd(model_na(md) * stride * 8);
        if (integrator == EP_INTEGRATOR_AB2) b += rnd(kHistSlots * stride * r);
    }
    return b;
}

// Upload (or rebuild) the job's conduction graph for its current
// parameters: state arrays at rest, FV coefficients, junction tables, and
// the junction flags in the cells' parameter-set bytes.
int graph_apply(ep_job *job) {
    ep_context *ctx = job->ctx;
    GraphPlan &g = *job->gp;
    const HostMesh &m = job->mesh();
    const int prec = job->precision;
    const size_t r = prec == EP_FP64_PLAIN ? 8 : 4;
    cudaStreamSynchronize(ctx->stream);
    drop_plans_with(ctx, job);
    for (auto &b : job->gbufs) dfree(ctx, &b);
    job->gbufs.clear();
    dfree(ctx, &job->graph_view);
    DevGraph G{};
    const int64_t n = g.n;
    int rc = EP_OK;
    void *q = nullptr;
    auto grab = [&](size_t bytes, void **dst) {
        DevBuf b;
        int r2 = dalloc(ctx, bytes, &b);
        if (!r2) {
            job->gbufs.push_back(b);
            *dst = b.p;
        }
        return r2;
    };
    auto put = [&](auto &vec, void **dst) { return upload(ctx, vec, &job->gbufs, dst); };
    G.n_nodes = n;
    for (int k = 0; k < 2 && !rc; ++k) rc = grab(std::max<int64_t>(n, 1) * r, &G.V[k]);
    for (int k = 0; k < 2 && !rc; ++k) rc = grab(std::max<int64_t>(n, 1) * r, &G.W[k]);
    if (!rc) rc = grab(std::max<int64_t>(n, 1) * r, &G.itot);
    if (!rc) rc = grab(std::max<int64_t>(n, 1) * r, &G.act);
    if (!rc) rc = put(g.row, &q), G.row = static_cast<const int *>(q);
    if (!rc) rc = put(g.col, &q), G.col = static_cast<const int *>(q);
    if (!rc) {
        if (prec == EP_FP64_PLAIN) rc = put(g.coef, &q);
        else {
            std::vector<float> f(g.coef.begin(), g.coef.end());
            rc = put(f, &q);
        }
        G.coef = q;
    }
    if (!rc) rc = put(g.pset, &q), G.pset = static_cast<const uint8_t *>(q);
    if (!rc) rc = put(g.smask, &q), G.smask = static_cast<const uint8_t *>(q);
    for (int md = 0; md < EP_N_MODELS && !rc; ++md) {
        DevRegion &rg = G.reg[md];
        rg.off = g.model_off[md];
        rg.n = g.model_off[md + 1] - g.model_off[md];
        rg.stride = round_up(std::max<int64_t>(rg.n, 1), 64);
        rg.r = nullptr;
        rg.a = nullptr;
        if (rg.n == 0) continue;
        rc = grab(size_t(model_nr(md)) * rg.stride * r, &rg.r);
        if (!rc) rc = grab(size_t(model_na(md)) * rg.stride * 8, &q), rg.a = static_cast<double *>(q);
    }
    const int64_t nj = int64_t(g.jnode.size());
    G.n_junc = int(nj);
    if (!rc) rc = put(g.jnode, &q), G.jnode = static_cast<const int *>(q);
    if (!rc) rc = put(g.jcell, &q), G.jcell = static_cast<const int *>(q);
    if (!rc) rc = put(g.jmode, &q), G.jmode = static_cast<const uint8_t *>(q);
    std::vector<double> neg(std::max<int64_t>(nj, 1), -INFINITY);
    if (!rc) rc = put(neg, &q), G.t_graph = static_cast<double *>(q);
    if (!rc) rc = put(neg, &q), G.t_cell = static_cast<double *>(q);
    if (!rc) rc = put(g.node_junc_ptr, &q), G.node_junc_ptr = static_cast<const int *>(q);
    if (!rc) rc = put(g.node_junc, &q), G.node_junc = static_cast<const int *>(q);
    if (!rc) rc = put(g.tgt_cell, &q), G.tgt_cell = static_cast<const int *>(q);
    if (!rc) rc = put(g.tgt_junc, &q), G.tgt_junc = static_cast<const int *>(q);
    if (!rc) rc = put(g.new2old, &q), job->gperm_dev = static_cast<const int *>(q);
    if (rc) return rc;
    G.n_tgt = int(g.tgt_cell.size());
    G.two_way = g.p.two_way;
    G.cell_nodes = 0;
    for (uint8_t md : g.jmode) G.cell_nodes |= md == EP_PMJ_CELL;
    G.substeps = g.substeps = std::max(1, int(std::ceil(job->params.dt * g.rho / 1.8)));
    G.g_graph = g.p.g_graph;
    G.g_cell = g.p.g_cell;
    G.threshold = g.p.threshold;
    G.delay_ortho = g.p.delay_ortho;
    G.delay_anti = g.p.delay_anti;
    G.amplitude = g.p.amplitude;
    G.duration = g.p.duration;
    G.h = job->params.dt / g.substeps;
    G.g_graph_f = float(G.g_graph);
    G.g_cell_f = float(G.g_cell);
    G.amplitude_f = float(G.amplitude);
    G.h_f = float(G.h);
    job->dj.g = G;
    // junction flags in the cells' parameter-set bytes
    std::vector<uint8_t> ps(m.pset);
    for (int32_t c : g.tgt_cell) ps[c] |= uint8_t(kJunctionFlag);
    cudaError_t e = cudaMemcpyAsync(const_cast<uint8_t *>(job->dj.pset), ps.data(), ps.size(), cudaMemcpyHostToDevice,
                                    ctx->upload);
    if (e == cudaSuccess) e = cudaMemcpyAsync(job->dj_dev.p, &job->dj, sizeof(DevJob), cudaMemcpyHostToDevice, ctx->upload);
    // the graph view: a DevJob whose cells are the graph nodes, for init and state transfer
    DevJob view = job->dj;
    view.V[0] = G.V[0];
    view.V[1] = G.V[1];
    view.act = G.act;
    view.n_cells = n;
    for (int md = 0; md < EP_N_MODELS; ++md) view.reg[md] = G.reg[md];
    view.pset = G.pset;
    if (e == cudaSuccess && (rc = dalloc(ctx, sizeof(DevJob), &job->graph_view))) return rc;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(job->graph_view.p, &view, sizeof(DevJob), cudaMemcpyHostToDevice, ctx->upload);
    if (e == cudaSuccess && n > 0)
        e = launch_init(prec, static_cast<const DevJob *>(job->graph_view.p), n, ctx->upload);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph upload");
    job->graph_tiles.clear();
    for (int md = 0; md < EP_N_MODELS; ++md)
        for (int64_t s = g.model_off[md]; s < g.model_off[md + 1]; s += kGraphThreads)
            job->graph_tiles.push_back(
                Tile{0, md, int(s), int(std::min<int64_t>(kGraphThreads, g.model_off[md + 1] - s))});
    // local tables of the one-launch substeps: each tile's nodes, then every node within
    // `substeps` hops of them (breadth first), with the neighbours as local indices
    {
        std::vector<int> lt_ptr{0}, lcol, mark(size_t(std::max<int64_t>(n, 1)), -1), nodes;
        std::vector<int2> lslot;
        int lmax = 0;
        for (const Tile &tl : job->graph_tiles) {
            nodes.clear();
            for (int i = 0; i < tl.count; ++i) {
                nodes.push_back(tl.start + i);
                mark[tl.start + i] = i;
            }
            size_t from = 0;
            for (int hop = 0; hop < g.substeps; ++hop) {
                const size_t to = nodes.size();
                for (size_t q = from; q < to; ++q)
                    for (int e = g.row[nodes[q]]; e < g.row[nodes[q] + 1]; ++e)
                        if (mark[g.col[e]] < 0) {
                            mark[g.col[e]] = int(nodes.size());
                            nodes.push_back(g.col[e]);
                        }
                from = to;
            }
            for (int u : nodes) {
                lslot.push_back(make_int2(u, int(lcol.size())));
                for (int e = g.row[u]; e < g.row[u + 1]; ++e) lcol.push_back(mark[g.col[e]]);
            }
            for (int u : nodes) mark[u] = -1;
            lt_ptr.push_back(int(lslot.size()));
            lmax = std::max(lmax, int(nodes.size()));
        }
        if (lcol.empty()) lcol.push_back(-1);
        if (lslot.empty()) lslot.push_back(make_int2(0, 0));
        DevGraph &DG = job->dj.g;
        if (!rc) rc = put(lt_ptr, &q), DG.lt_ptr = static_cast<const int *>(q);
        if (!rc) rc = put(lslot, &q), DG.lslot = static_cast<const int2 *>(q);
        if (!rc) rc = put(lcol, &q), DG.lcol = static_cast<const int *>(q);
        if (rc) return rc;
        DG.lmax = lmax;
        job->graph_lmax = lmax;
        e = cudaMemcpyAsync(job->dj_dev.p, &job->dj, sizeof(DevJob), cudaMemcpyHostToDevice, ctx->upload);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph upload");
    }
    job->version++;
    for (auto &b : job->gbufs) job->device_bytes += b.bytes;
    return EP_OK;
}

// Upload (or rebuild) the bidomain state of a job for its current
// parameters and precision: the operator of D_i + D_e folded like the job's
// own, the gauge weights, v_e = 0 and the solver buffers; then solve v_e from
// the current V. The cell update adds L_i(v_e) from the next step on.
int bido_apply(ep_job *job) {
    ep_context *ctx = job->ctx;
    BidoHost &B = *job->bido;
    const HostMesh &m = job->mesh();
    const int prec = job->precision;
    const size_t r = prec == EP_FP64_PLAIN ? 8 : 4;
    const int64_t N = m.n_cells;
    cudaStreamSynchronize(ctx->stream);
    drop_plans_with(ctx, job);
    free_job_arrays(job, &B.bufs);
    ep_params p2 = job->params;
    for (int k = 0; k < p2.n_sets; ++k) {
        p2.sets[k].D_l += B.De_l[k];
        p2.sets[k].D_t += B.De_t[k];
    }
    Coeffs cf;
    std::string err;
    int rc = build_coeffs(m, &p2, &cf, &err);
    if (rc) return fail(ctx, rc, "ep_bidomain_enable: " + err);
    // gauge weights V_c / sum V
    std::vector<double> wv(N);
    double tot = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        const double *x0 = &m.xyz[3 * int64_t(m.tet[4 * c])];
        double d[3][3];
        for (int k = 1; k < 4; ++k)
            for (int a = 0; a < 3; ++a) d[k - 1][a] = m.xyz[3 * int64_t(m.tet[4 * c + k]) + a] - x0[a];
        const double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                           d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                           d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
        wv[c] = std::fabs(det) / 6.0;
        tot += wv[c];
    }
    for (auto &x : wv) x /= tot;
    auto put_r = [&](const std::vector<double> &v, const void **dst) -> int {
        void *q = nullptr;
        int r2;
        if (prec == EP_FP64_PLAIN) {
            r2 = upload(ctx, v, &B.bufs, &q);
        } else {
            std::vector<float> f(v.begin(), v.end());
            r2 = upload(ctx, f, &B.bufs, &q);
        }
        *dst = q;
        return r2;
    };
    auto grab = [&](size_t bytes, void **dst) {
        DevBuf b;
        int r2 = dalloc(ctx, bytes, &b);
        if (!r2) {
            B.bufs.push_back(b);
            *dst = b.p;
        }
        return r2;
    };
    BidoArgs a{};
    B.grid = bido_grid(prec, ctx->sm_count, N);
    a.ld = round_up(std::max<int64_t>(N, 1), 64);
    void *ve = nullptr, *xd = nullptr, *bb = nullptr, *w = nullptr, *basis = nullptr, *part = nullptr, *st = nullptr,
         *sy = nullptr;
    if (!rc) rc = put_r(cf.wa, &a.wa);
    if (!rc) rc = put_r(cf.wb, &a.wb);
    if (!rc) rc = put_r(cf.q, &a.q);
    if (!rc) rc = put_r(wv, &a.wvol);
    if (!rc) rc = grab(a.ld * r, &ve);
    if (!rc) rc = grab(N * r, &xd);
    if (!rc) rc = grab(N * r, &bb);
    if (!rc) rc = grab(a.ld * r, &w);
    if (!rc) rc = grab(size_t(B.restart + 1) * a.ld * r, &basis);
    void *vprev = nullptr;
    if (!rc) rc = grab(a.ld * r, &vprev);
    if (!rc) rc = grab(2 * size_t(kBidoMaxRestart + 1) * B.grid * sizeof(double), &part);
    if (!rc) rc = grab(sizeof(BidoStats), &st);
    if (!rc) rc = grab(sizeof(BidoSync), &sy);
    if (rc) {
        free_job_arrays(job, &B.bufs);
        return rc;
    }
    a.ve = ve;
    a.xdiv = xd;
    a.b = bb;
    a.w = w;
    a.basis = basis;
    a.vprev = vprev;
    a.part = static_cast<double *>(part);
    a.stats = static_cast<BidoStats *>(st);
    a.sync = static_cast<BidoSync *>(sy);
    a.tol = B.tol;
    a.atol = B.atol;
    a.max_iter = B.max_iter;
    a.restart = B.restart;
    a.mode = 0;
    a.reorth = B.reorth;
    a.barrier_limit_ns = static_cast<unsigned long long>(B.barrier_limit_s * 1e9);
    B.args = a;
    job->dj.xdiv = xd;
    // v_e = 0; the vector pads past n_cells must stay zero for the basis passes
    cudaError_t e = cudaMemsetAsync(ve, 0, a.ld * r, ctx->upload);
    if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, a.ld * r, ctx->upload);
    if (e == cudaSuccess) e = cudaMemsetAsync(basis, 0, size_t(B.restart + 1) * a.ld * r, ctx->upload);
    if (e == cudaSuccess) e = cudaMemsetAsync(vprev, 0, a.ld * r, ctx->upload);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(BidoStats), ctx->upload);
    if (e == cudaSuccess) e = cudaMemsetAsync(sy, 0, sizeof(BidoSync), ctx->upload);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(job->dj_dev.p, &job->dj, sizeof(DevJob), cudaMemcpyHostToDevice, ctx->upload);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload);
    if (e == cudaSuccess) e = launch_bido(prec, a, job->dj, B.grid, ctx->stream);   // v_e from the current V
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bidomain upload");
    job->version++;
    job->device_bytes = 0;
    for (auto *pool : {&job->topo, &job->prec, &job->gbufs, &B.bufs})
        for (auto &b : *pool) job->device_bytes += b.bytes;
    return EP_OK;
}

// AB2 keeps the previous step's rates; after the state or the step index is
// set from outside they are stale, so the next step is forward Euler again.
int restart_ab2(ep_job *job) {
    if (!job->has_params || job->params.integrator != EP_INTEGRATOR_AB2) return EP_OK;
    ep_context *ctx = job->ctx;
    long long cur = 0;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&cur, job->step_dev.p, sizeof(cur), cudaMemcpyDeviceToHost);
    job->dj.ab2_from = cur;
    if (e == cudaSuccess) e = cudaMemcpy(job->dj_dev.p, &job->dj, sizeof(DevJob), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "AB2 restart");
    job->version++;   // the plans' copies of the job descriptor are rebuilt
    return EP_OK;
}

// Back to the monodomain model (also the cleanup of a failed bido_apply).
void bido_drop(ep_job *job) {
    ep_context *ctx = job->ctx;
    if (!job->bido) return;
    cudaStreamSynchronize(ctx->stream);
    drop_plans_with(ctx, job);
    for (auto &b : job->bido->bufs) job->device_bytes -= b.bytes;
    free_job_arrays(job, &job->bido->bufs);
    job->bido.reset();
    job->dj.xdiv = nullptr;
    cudaMemcpyAsync(job->dj_dev.p, &job->dj, sizeof(DevJob), cudaMemcpyHostToDevice, ctx->upload);
    cudaStreamSynchronize(ctx->upload);
    job->version++;
}

}  // namespace

struct ep_plan {
    std::shared_ptr<HostMesh> mesh;
    std::shared_ptr<Sell> sell;
    bool has_params = false;
    ep_params params{};
    Coeffs cf;
};

extern "C" {

int ep_mesh_create(ep_context *ctx, const ep_mesh_desc *desc, ep_job **out) {
    if (!ctx || !desc || !out) return fail(ctx, EP_EINVAL, "ep_mesh_create: NULL argument");
    DeviceGuard g(ctx->device);
    try {
        std::unique_ptr<ep_job> j(new ep_job());
        j->ctx = ctx;
        auto mesh = std::make_shared<HostMesh>();
        std::string err;
        int rc = build_mesh(desc, mesh.get(), &err);
        if (rc) return fail(ctx, rc, err);
        auto sell = std::make_shared<Sell>();
        build_sell(*mesh, sell.get());
        j->mp = mesh;
        j->sp = sell;
        if ((rc = job_upload_topology(ctx, j.get()))) {
            free_job_arrays(j.get(), &j->topo);
            dfree(ctx, &j->dj_dev);
            dfree(ctx, &j->step_dev);
            return rc;
        }
        ctx->jobs.insert(j.get());
        *out = j.release();
        return EP_OK;
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_mesh_create: out of host memory");
    }
}

int ep_params_set(ep_job *job, const ep_params *p) {
    if (!job || !p) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    DeviceGuard g(ctx->device);
    try {
        std::string err;
        Coeffs cf;
        int rc = plan_params(job->mesh(), p, &cf, &err);
        if (rc) return fail(ctx, rc, "ep_params_set: " + err);
        return job_apply_params(job, p, cf);
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_params_set: out of host memory");
    }
}

int ep_plan_create(const ep_mesh_desc *desc, const ep_params *params, ep_plan **out) {
    if (!desc || !out) {
        g_create_error = "ep_plan_create: NULL argument";
        return EP_EINVAL;
    }
    try {
        std::unique_ptr<ep_plan> pl(new ep_plan());
        pl->mesh = std::make_shared<HostMesh>();
        std::string err;
        int rc = build_mesh(desc, pl->mesh.get(), &err);
        if (!rc) {
            pl->sell = std::make_shared<Sell>();
            build_sell(*pl->mesh, pl->sell.get());
            if (params) {
                rc = plan_params(*pl->mesh, params, &pl->cf, &err);
                pl->has_params = rc == EP_OK;
                pl->params = *params;
            }
        }
        if (rc) {
            g_create_error = "ep_plan_create: " + err;
            return rc;
        }
        *out = pl.release();
        return EP_OK;
    } catch (const std::bad_alloc &) {
        g_create_error = "ep_plan_create: out of host memory";
        return EP_ENOMEM;
    }
}

int64_t ep_plan_bytes(const ep_plan *plan) {
    if (!plan) return -1;
    return job_bytes(*plan->mesh, *plan->sell, plan->has_params ? plan->params.precision : EP_FP32_MIXED,
                     plan->has_params ? plan->params.integrator : EP_INTEGRATOR_FE);
}

int ep_plan_info(const ep_plan *plan, int64_t *n_cells, int64_t *n_nodes, int32_t *index_width,
                 int32_t *node_index_width) {
    if (!plan) return EP_EINVAL;
    if (n_cells) *n_cells = plan->mesh->n_cells;
    if (n_nodes) *n_nodes = plan->mesh->n_nodes;
    if (index_width) *index_width = plan->sell->idx16 ? 16 : 32;
    if (node_index_width) *node_index_width = plan->sell->col16ok ? 16 : 32;
    return EP_OK;
}

int ep_plan_destroy(ep_plan *plan) {
    delete plan;
    return EP_OK;
}

int ep_job_create(ep_context *ctx, const ep_plan *plan, ep_job **out) {
    if (!ctx || !plan || !out) return fail(ctx, EP_EINVAL, "ep_job_create: NULL argument");
    DeviceGuard g(ctx->device);
    try {
        std::unique_ptr<ep_job> j(new ep_job());
        j->ctx = ctx;
        j->mp = plan->mesh;
        j->sp = plan->sell;
        int rc = job_upload_topology(ctx, j.get());
        if (!rc && plan->has_params) rc = job_apply_params(j.get(), &plan->params, plan->cf);
        if (rc) {
            free_job_arrays(j.get(), &j->prec);
            free_job_arrays(j.get(), &j->topo);
            dfree(ctx, &j->dj_dev);
            dfree(ctx, &j->step_dev);
            return rc;
        }
        ctx->jobs.insert(j.get());
        *out = j.release();
        return EP_OK;
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_job_create: out of host memory");
    }
}

// The launch groups of a batch: the FP64 jobs in one group; the FP32 jobs
// that step by forward Euler without the bidomain solve in groups of at most
// kParamJobs (their kernels take the group's descriptors as a parameter),
// the other FP32 jobs in one group.
static std::vector<std::pair<int, std::vector<int>>> launch_groups(ep_job *const *jobs, int n) {
    std::vector<std::pair<int, std::vector<int>>> out;
    std::vector<int> f64, plain, other;
    for (int i = 0; i < n; ++i) {
        if (jobs[i]->precision == EP_FP64_PLAIN) f64.push_back(i);
        else if (jobs[i]->params.integrator == EP_INTEGRATOR_AB2 || jobs[i]->bido) other.push_back(i);
        else plain.push_back(i);
    }
    for (size_t a = 0; a < plain.size(); a += kParamJobs)
        out.push_back({EP_FP32_MIXED, std::vector<int>(plain.begin() + a,
                                                       plain.begin() + std::min(plain.size(), a + kParamJobs))});
    if (!other.empty()) out.push_back({EP_FP32_MIXED, other});
    if (!f64.empty()) out.push_back({EP_FP64_PLAIN, f64});
    return out;
}

static int build_plan(ep_context *ctx, ep_job *const *jobs, int n, Plan *pl) {
    pl->jobs.assign(jobs, jobs + n);
    for (int i = 0; i < n; ++i) pl->versions.push_back(jobs[i]->version);
    for (const auto &grp : launch_groups(jobs, n)) {
        const int prec = grp.first;
        std::vector<DevJob> tab;
        std::vector<Tile> nt, ct, gt, gst;
        std::vector<Work> wk;
        std::vector<int> cell_begin, node_begin;   // first tile of each job
        int max_lmax = 0;
        int max_sub = 0, any_bido = 0, any_ab2 = 0, n_idx16 = 0, n_col16 = 0, models = 0;
        for (int i : grp.second) {
            const int jid = int(tab.size());
            tab.push_back(jobs[i]->dj);
            append_work(jobs[i], int(nt.size()), int(ct.size()), &wk);
            cell_begin.push_back(int(ct.size()));
            node_begin.push_back(int(nt.size()));
            for (Tile t : jobs[i]->node_tiles) nt.push_back(Tile{jid, t.model, t.start, t.count});
            for (Tile t : jobs[i]->cell_tiles) ct.push_back(Tile{jid, t.model, t.start, t.count});
            if (jobs[i]->params.integrator == EP_INTEGRATOR_AB2) any_ab2 = 1;
            if (jobs[i]->dj.idx16) ++n_idx16;
            if (jobs[i]->dj.col16) ++n_col16;
            for (int m = 0; m < EP_N_MODELS; ++m)
                if (jobs[i]->mesh().model_off[m + 1] > jobs[i]->mesh().model_off[m]) models |= 1 << m;
            if (jobs[i]->bido) {
                any_bido = 1;
                pl->bido.push_back(jobs[i]);
            }
            if (jobs[i]->gp) {
                int k = 0;
                for (Tile t : jobs[i]->graph_tiles) {
                    gt.push_back(Tile{jid, t.model, t.start, t.count});
                    gst.push_back(Tile{jid, k++, t.start, t.count});
                }
                max_sub = std::max(max_sub, jobs[i]->gp->substeps);
                max_lmax = std::max(max_lmax, jobs[i]->graph_lmax);
            }
        }
        if (tab.empty()) continue;
        Plan::Group g{};
        g.precision = prec;
        g.n_jobs = int(tab.size());
        std::vector<DevBuf> tmp;
        void *p;
        int rc;
        if ((rc = upload(ctx, tab, &tmp, &p))) return rc;
        g.jobtab = tmp.back();
        if ((rc = upload(ctx, nt, &tmp, &p))) return rc;
        g.node_tiles = tmp.back();
        if ((rc = upload(ctx, ct, &tmp, &p))) return rc;
        g.cell_tiles = tmp.back();
        if ((rc = upload(ctx, wk, &tmp, &p))) return rc;
        g.work = tmp.back();
        // [0] the cell launch's ticket, [1] the fused launch's work counter
        if ((rc = dalloc(ctx, 2 * sizeof(unsigned), &g.done))) return rc;
        cudaMemsetAsync(g.done.p, 0, 2 * sizeof(unsigned), ctx->upload);
        g.L.work = static_cast<const Work *>(g.work.p);
        g.L.n_work = int(wk.size());
        g.L.head = static_cast<unsigned *>(g.done.p) + 1;
        g.L.jobs = static_cast<const DevJob *>(g.jobtab.p);
        g.L.n_jobs = g.n_jobs;
        g.L.node_tiles = static_cast<const Tile *>(g.node_tiles.p);
        g.L.n_node_tiles = int(nt.size());
        g.L.cell_tiles = static_cast<const Tile *>(g.cell_tiles.p);
        g.L.n_cell_tiles = int(ct.size());
        g.L.done = static_cast<unsigned *>(g.done.p);
        g.L.graph_tiles = nullptr;
        g.L.n_graph_tiles = 0;
        g.L.graph_substeps = 0;
        g.L.graph_grid = 1;
        g.L.bido = any_bido;
        g.L.ab2 = any_ab2;
        g.L.idx16 = n_idx16 > 0;
        g.L.sm_count = ctx->sm_count;
        g.L.node_form = n_col16 == 0 ? 0 : (n_col16 == g.n_jobs ? 1 : 2);
        g.L.models = models;
        g.L.err = static_cast<unsigned *>(ctx->err_word.p);
        if (!gt.empty()) {
            if ((rc = upload(ctx, gt, &tmp, &p))) return rc;
            g.graph_tiles = tmp.back();
            g.L.graph_tiles = static_cast<const Tile *>(g.graph_tiles.p);
            g.L.n_graph_tiles = int(gt.size());
            g.L.graph_substeps = max_sub;
            if ((rc = upload(ctx, gst, &tmp, &p))) return rc;
            g.graph_sub_tiles = tmp.back();
            g.L.graph_sub_tiles = static_cast<const Tile *>(g.graph_sub_tiles.p);
            g.L.graph_lmax = max_lmax;
            g.L.graph_local = ctx->graph_mode == EP_GRAPH_SUBSTEPS_LOCAL;
            g.L.graph_grid = std::max(1, std::min<int>(int(gt.size()), ctx->sm_count * 4));
        }
        g.L.node_grid = std::max(1, std::min<int>(int(nt.size()), ctx->sm_count * node_blocks_per_sm(prec)));
        g.L.cell_variant = ctx->cell_variant[prec];
        g.L.cell_grid0 = std::max(1, std::min<int>(int(ct.size()), ctx->sm_count * cell_blocks_per_sm(prec, 0)));
        g.L.cell_grid =
            std::max(1, std::min<int>(int(ct.size()), ctx->sm_count * cell_blocks_per_sm(prec, g.L.cell_variant)));
        cell_begin.push_back(int(ct.size()));
        node_begin.push_back(int(nt.size()));
        auto fill = [&](auto &jt) {
            jt.n_jobs = g.n_jobs;
            for (int k = 0; k <= g.n_jobs; ++k) {
                jt.cell_begin[k] = cell_begin[k];
                jt.node_begin[k] = node_begin[k];
            }
            for (int k = 0; k < g.n_jobs; ++k) jt.j[k] = tab[k];
        };
        if (g.n_jobs == 1) {
            g.tab1 = std::make_shared<JobTab<1>>();
            fill(*g.tab1);
            g.L.tab1 = g.tab1.get();
        } else if (g.n_jobs <= kParamJobs) {
            g.tabk = std::make_shared<JobTab<kParamJobs>>();
            fill(*g.tabk);
            g.L.tabk = g.tabk.get();
        }
        pl->groups.push_back(g);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->upload);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "plan");
}

static cudaError_t enqueue_steps(Plan *pl, int64_t steps, cudaStream_t s) {
    for (int64_t it = 0; it < steps; ++it) {
        for (auto &g : pl->groups) {
            cudaError_t e = launch_step(g.precision, g.L, s);
            if (e != cudaSuccess) return e;
        }
        for (ep_job *j : pl->bido) {   // second line of Eq. 6 for v_e^{n+1}
            cudaError_t e = launch_bido(j->precision, j->bido->args, j->dj, j->bido->grid, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

static int check_jobs(ep_job *const *jobs, int32_t n_jobs, int64_t n_steps, const char *who) {
    ep_context *ctx = jobs[0]->ctx;
    if (n_steps < 0) return fail(ctx, EP_EINVAL, std::string(who) + ": n_steps < 0");
    for (int i = 0; i < n_jobs; ++i) {
        if (!jobs[i] || jobs[i]->ctx != ctx) return fail(ctx, EP_EINVAL, std::string(who) + ": jobs of different contexts");
        if (!jobs[i]->has_params) return fail(ctx, EP_ESTATE, std::string(who) + ": a job has no parameters");
        for (int k = 0; k < i; ++k)
            if (jobs[k] == jobs[i]) return fail(ctx, EP_EINVAL, std::string(who) + ": job listed twice");
    }
    return EP_OK;
}

// The cached plan (job tables, tiles, graph) of this exact job list, built on first use.
static int get_plan(ep_context *ctx, ep_job *const *jobs, int32_t n_jobs, Plan **out) {
    for (size_t k = 0; k < ctx->plans.size(); ++k) {
        Plan *p = ctx->plans[k].get();
        if (int(p->jobs.size()) != n_jobs || !std::equal(p->jobs.begin(), p->jobs.end(), jobs)) continue;
        bool same = true;
        for (int i = 0; i < n_jobs; ++i) same = same && p->versions[i] == jobs[i]->version;
        if (same) {
            *out = p;
            return EP_OK;
        }
        free_plan(ctx, p);
        ctx->plans.erase(ctx->plans.begin() + k);
        break;
    }
    std::unique_ptr<Plan> np(new Plan());
    int rc = build_plan(ctx, jobs, n_jobs, np.get());
    if (rc) {
        free_plan(ctx, np.get());
        return rc;
    }
    if (ctx->plans.size() >= kMaxPlans) {
        cudaStreamSynchronize(ctx->stream);   // its tables may still be read by queued steps
        free_plan(ctx, ctx->plans.front().get());
        ctx->plans.erase(ctx->plans.begin());
    }
    ctx->plans.push_back(std::move(np));
    *out = ctx->plans.back().get();
    return EP_OK;
}

int ep_step(ep_job *const *jobs, int32_t n_jobs, int64_t n_steps) {
    if (!jobs || n_jobs <= 0 || !jobs[0]) return EP_EINVAL;
    ep_context *ctx = jobs[0]->ctx;
    int rc = check_jobs(jobs, n_jobs, n_steps, "ep_step");
    if (rc) return rc;
    // a staged cell kernel of an earlier call gave up waiting for its copies (the word is
    // read back asynchronously after each call that ran one)
    if (*ctx->err_host)
        return fail(ctx, EP_ETIMEOUT, "ep_step: an earlier step's bounded wait gave up (staged copies or fused "
                                      "node tiles); the state of the jobs stepped since is undefined (restore a "
                                      "checkpoint, then ep_clear_error)");
    if (n_steps == 0) return EP_OK;
    DeviceGuard g(ctx->device);
    try {
        Plan *pl = nullptr;
        if ((rc = get_plan(ctx, jobs, n_jobs, &pl))) return rc;
        bool staged = false;   // staged or fused: kernels with bounded waits that report through the error word
        for (auto &gr : pl->groups)
            staged = staged || is_staged_variant(gr.L.cell_variant) || is_fused_variant(gr.L.cell_variant);
        int64_t left = n_steps;
        if (n_steps >= kGraphMinSteps && pl->bido.empty()) {   // cooperative solves launch directly
            if (!pl->exec) {
                cudaError_t e = cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e2 = enqueue_steps(pl, kGraphSteps, ctx->capture);
                    e = cudaStreamEndCapture(ctx->capture, &pl->graph);
                    if (e2 != cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_step: graph capture");
            }
            for (; left >= kGraphSteps; left -= kGraphSteps) {
                cudaError_t e = cudaGraphLaunch(pl->exec, ctx->stream);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_step: graph launch");
            }
        }
        cudaError_t e = enqueue_steps(pl, left, ctx->stream);
        if (e == cudaSuccess && staged)
            e = cudaMemcpyAsync(ctx->err_host, ctx->err_word.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_step: launch");
        return EP_OK;
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_step: out of host memory");
    }
}

int ep_time_kernels(ep_job *const *jobs, int32_t n_jobs, int64_t n_steps, double *node_ms, double *cell_ms) {
    if (!jobs || n_jobs <= 0 || !jobs[0] || !node_ms || !cell_ms) return EP_EINVAL;
    ep_context *ctx = jobs[0]->ctx;
    int rc = check_jobs(jobs, n_jobs, n_steps, "ep_time_kernels");
    if (rc) return rc;
    *node_ms = *cell_ms = 0.0;
    if (n_steps == 0) return EP_OK;
    DeviceGuard g(ctx->device);
    try {
        Plan *pl = nullptr;
        if ((rc = get_plan(ctx, jobs, n_jobs, &pl))) return rc;
        const size_t ng = pl->groups.size();
        std::vector<cudaEvent_t> ev(3 * ng * n_steps, nullptr);
        cudaError_t e = cudaSuccess;
        for (auto &x : ev)
            if (e == cudaSuccess) e = cudaEventCreate(&x);
        size_t k = 0;
        for (int64_t it = 0; it < n_steps && e == cudaSuccess; ++it)
            for (auto &gr : pl->groups) {
                e = cudaEventRecord(ev[k++], ctx->stream);
                if (e == cudaSuccess) e = launch_node(gr.precision, gr.L, ctx->stream);
                if (e == cudaSuccess) e = launch_graph(gr.precision, gr.L, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev[k++], ctx->stream);
                if (e == cudaSuccess) e = launch_cell(gr.precision, gr.L, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev[k++], ctx->stream);
            }
            for (ep_job *j : pl->bido)   // untimed: the elliptic solves of bidomain jobs
                if (e == cudaSuccess) e = launch_bido(j->precision, j->bido->args, j->dj, j->bido->grid, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        double tn = 0.0, tc = 0.0;
        for (size_t i = 0; i + 2 < k + 1 && e == cudaSuccess; i += 3) {
            float a = 0.f, b = 0.f;
            e = cudaEventElapsedTime(&a, ev[i], ev[i + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[i + 1], ev[i + 2]);
            tn += a;
            tc += b;
        }
        for (auto &x : ev)
            if (x) cudaEventDestroy(x);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_time_kernels");
        *node_ms = tn / double(n_steps);
        *cell_ms = tc / double(n_steps);
        return EP_OK;
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_time_kernels: out of host memory");
    }
}

// Use launch shape `variant` for the cell kernel of `precision` in every plan
// of the context (captured graphs are re-captured on next use).
static void apply_cell_variant(ep_context *ctx, int precision, int variant) {
    ctx->cell_variant[precision] = variant;
    for (auto &p : ctx->plans) {
        bool touched = false;
        for (auto &g : p->groups)
            if (g.precision == precision) {
                g.L.cell_variant = variant;
                g.L.cell_grid = std::max(1, std::min<int>(g.L.n_cell_tiles,
                                                          ctx->sm_count * cell_blocks_per_sm(precision, variant)));
                touched = true;
            }
        if (touched) {
            if (p->exec) cudaGraphExecDestroy(p->exec);
            if (p->graph) cudaGraphDestroy(p->graph);
            p->exec = nullptr;
            p->graph = nullptr;
        }
    }
}

int ep_alu_peaks(ep_context *ctx, double *out) {
    if (!ctx || !out) return EP_EINVAL;
    DeviceGuard g(ctx->device);
    DevBuf sink;
    int rc = dalloc(ctx, 16, &sink);
    if (rc) return rc;
    // iterations per kind: about a millisecond per launch on a full B300
    const int iters[3] = {16384, 2048, 512};
    const int blocks = ctx->sm_count * (2048 / alu_probe_threads());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
        double ops = 0.0, best = 0.0;
        e = launch_alu_probe(kind, blocks, iters[kind], static_cast<double *>(sink.p), ctx->stream, &ops);  // warm-up
        for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, ctx->stream);
            if (e == cudaSuccess) e = launch_alu_probe(kind, blocks, iters[kind], static_cast<double *>(sink.p), ctx->stream, &ops);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms > 0.f) best = std::max(best, ops / (1e-3 * double(ms)));
        }
        out[kind] = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_alu_peaks");
    return EP_OK;
}

int ep_set_cell_variant(ep_context *ctx, int32_t precision, int32_t variant) {
    if (!ctx) return EP_EINVAL;
    if ((precision != EP_FP32_MIXED && precision != EP_FP64_PLAIN) || variant < 0 || variant >= kNumCellVariants)
        return fail(ctx, EP_EINVAL, "ep_set_cell_variant: unknown precision or variant");
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    apply_cell_variant(ctx, precision, variant);
    return EP_OK;
}

int ep_autotune(ep_job *const *jobs, int32_t n_jobs, int32_t steps_per_variant, int32_t *chosen, double *variant_ms) {
    if (!jobs || n_jobs <= 0 || !jobs[0] || steps_per_variant <= 0) return EP_EINVAL;
    ep_context *ctx = jobs[0]->ctx;
    int rc = check_jobs(jobs, n_jobs, 0, "ep_autotune");
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    try {
        Plan *pl = nullptr;
        if ((rc = get_plan(ctx, jobs, n_jobs, &pl))) return rc;
        cudaEvent_t e0, e1;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_autotune");
        for (int p = 0; p < 2; ++p) {
            if (chosen) chosen[p] = -1;
            for (int v = 0; v < kNumCellVariants && variant_ms; ++v) variant_ms[p * kNumCellVariants + v] = -1.0;
        }
        // per precision: every variant on all of that precision's launch groups at once, timing their
        // whole steps (node values, conduction graphs, cell update; the fused variants do the node
        // values in their one launch); the other precision's groups step untimed in between, so all
        // jobs stay in step
        for (int prec : {EP_FP32_MIXED, EP_FP64_PLAIN}) {
            bool any = false;
            for (auto &gr : pl->groups) any = any || gr.precision == prec;
            if (!any) continue;
            double best = 1e300;
            int best_v = 0;
            for (int v = 0; v < kNumCellVariants && e == cudaSuccess; ++v) {
                for (auto &gr : pl->groups)
                    if (gr.precision == prec) {
                        gr.L.cell_variant = v;
                        gr.L.cell_grid = std::max(1, std::min<int>(gr.L.n_cell_tiles,
                                                                   ctx->sm_count * cell_blocks_per_sm(prec, v)));
                    }
                double tot = 0.0;
                for (int it = 0; it < steps_per_variant && e == cudaSuccess; ++it) {
                    e = cudaEventRecord(e0, ctx->stream);
                    for (auto &gr : pl->groups) {
                        if (gr.precision != prec) continue;
                        if (e == cudaSuccess) e = launch_node(prec, gr.L, ctx->stream);
                        if (e == cudaSuccess) e = launch_graph(prec, gr.L, ctx->stream);
                        if (e == cudaSuccess) e = launch_cell(prec, gr.L, ctx->stream);
                    }
                    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    tot += ms;
                    for (auto &other : pl->groups)
                        if (other.precision != prec && e == cudaSuccess)
                            e = launch_step(other.precision, other.L, ctx->stream);
                    for (ep_job *j : pl->bido)
                        if (e == cudaSuccess) e = launch_bido(j->precision, j->bido->args, j->dj, j->bido->grid, ctx->stream);
                }
                const double mean = tot / steps_per_variant;
                if (variant_ms) variant_ms[prec * kNumCellVariants + v] = mean;
                if (mean < best) {
                    best = mean;
                    best_v = v;
                }
            }
            if (e != cudaSuccess) break;
            apply_cell_variant(ctx, prec, best_v);
            if (chosen) chosen[prec] = best_v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "ep_autotune");
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_autotune: out of host memory");
    }
}

static int check_io(ep_job *job, int64_t n, const void *buf) {
    if (!job) return EP_EINVAL;
    if (!buf || n != job->mesh().n_cells)
        return fail(job->ctx, EP_EINVAL, "buffer is NULL or its length differs from the number of cells");
    if (!job->has_params) return fail(job->ctx, EP_ESTATE, "job has no parameters (no state yet)");
    return EP_OK;
}

static int transfer_state(ep_job *job, int32_t model, int32_t var, double *host, int64_t n, bool write) {
    int rc = check_io(job, n, host);
    if (rc) return rc;
    ep_context *ctx = job->ctx;
    if (model < 0 || model >= EP_N_MODELS || var < 0 || var >= model_nvar(model))
        return fail(ctx, EP_EINVAL, "unknown model or variable id");
    DeviceGuard g(ctx->device);
    DevBuf b;
    if ((rc = dalloc(ctx, n * sizeof(double), &b))) return rc;
    cudaError_t e = cudaSuccess;
    const DevJob *dj = static_cast<const DevJob *>(job->dj_dev.p);
    double *buf = static_cast<double *>(b.p);
    if (write) {
        e = cudaMemcpyAsync(buf, host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_scatter(job->precision, dj, job->perm_dev, n, model, var, buf, ctx->stream);
    } else {
        e = launch_gather(job->precision, dj, job->perm_dev, n, model, var, buf, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, write ? "ep_write_state" : "ep_read_state");
    return write ? restart_ab2(job) : EP_OK;
}

int ep_read_state(ep_job *job, int32_t model, int32_t var, double *host_out, int64_t n) {
    try {
        return transfer_state(job, model, var, host_out, n, false);
    } catch (const std::bad_alloc &) {
        return fail(job->ctx, EP_ENOMEM, "ep_read_state: out of host memory");
    }
}

int ep_write_state(ep_job *job, int32_t model, int32_t var, const double *host_in, int64_t n) {
    try {
        return transfer_state(job, model, var, const_cast<double *>(host_in), n, true);
    } catch (const std::bad_alloc &) {
        return fail(job->ctx, EP_ENOMEM, "ep_write_state: out of host memory");
    }
}

// The same transfers in FP32, for jobs that compute in FP32 (EP_FP32_MIXED)
// and the variables they store in FP32: exact, with half the bytes.
static int transfer_state_f32(ep_job *job, int32_t model, int32_t var, float *host, int64_t n, bool write) {
    int rc = check_io(job, n, host);
    if (rc) return rc;
    ep_context *ctx = job->ctx;
    if (model < 0 || model >= EP_N_MODELS || var < 0 || var >= model_nvar(model))
        return fail(ctx, EP_EINVAL, "unknown model or variable id");
    if (job->precision != EP_FP32_MIXED)
        return fail(ctx, EP_EINVAL, "FP32 state transfers need an EP_FP32_MIXED job");
    if (model_vars(model)[var].kind == kVarA)
        return fail(ctx, EP_EINVAL, std::string(model_vars(model)[var].name) +
                                        " is stored as a compensated sum: use ep_read_state / ep_write_state");
    DeviceGuard g(ctx->device);
    DevBuf b;
    if ((rc = dalloc(ctx, n * sizeof(float), &b))) return rc;
    const DevJob *dj = static_cast<const DevJob *>(job->dj_dev.p);
    float *buf = static_cast<float *>(b.p);
    cudaError_t e = cudaSuccess;
    if (write) {
        e = cudaMemcpyAsync(buf, host, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_transfer_f32(dj, job->perm_dev, n, model, var, buf, 1, ctx->stream);
    } else {
        e = launch_transfer_f32(dj, job->perm_dev, n, model, var, buf, 0, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, write ? "ep_write_state_f32" : "ep_read_state_f32");
    return write ? restart_ab2(job) : EP_OK;
}

int ep_read_state_f32(ep_job *job, int32_t model, int32_t var, float *host_out, int64_t n) {
    try {
        return transfer_state_f32(job, model, var, host_out, n, false);
    } catch (const std::bad_alloc &) {
        return fail(job->ctx, EP_ENOMEM, "ep_read_state_f32: out of host memory");
    }
}

int ep_write_state_f32(ep_job *job, int32_t model, int32_t var, const float *host_in, int64_t n) {
    try {
        return transfer_state_f32(job, model, var, const_cast<float *>(host_in), n, true);
    } catch (const std::bad_alloc &) {
        return fail(job->ctx, EP_ENOMEM, "ep_write_state_f32: out of host memory");
    }
}

int ep_activation_times_f32(ep_job *job, float *host_out, int64_t n) {
    int rc = check_io(job, n, host_out);
    if (rc) return rc;
    ep_context *ctx = job->ctx;
    if (job->precision != EP_FP32_MIXED)
        return fail(ctx, EP_EINVAL, "FP32 activation times need an EP_FP32_MIXED job");
    DeviceGuard g(ctx->device);
    DevBuf b;
    if ((rc = dalloc(ctx, n * sizeof(float), &b))) return rc;
    cudaError_t e = launch_gather_act_f32(static_cast<const DevJob *>(job->dj_dev.p), job->perm_dev, n,
                                          static_cast<float *>(b.p), ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, b.p, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "ep_activation_times_f32");
}

int ep_activation_times(ep_job *job, double *host_out, int64_t n) {
    int rc = check_io(job, n, host_out);
    if (rc) return rc;
    ep_context *ctx = job->ctx;
    DeviceGuard g(ctx->device);
    DevBuf b;
    if ((rc = dalloc(ctx, n * sizeof(double), &b))) return rc;
    cudaError_t e = launch_gather_act(job->precision, static_cast<const DevJob *>(job->dj_dev.p), job->perm_dev, n,
                                      static_cast<double *>(b.p), ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, b.p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "ep_activation_times");
}

int ep_reset_activation(ep_job *job) {
    if (!job) return EP_EINVAL;
    if (!job->has_params) return fail(job->ctx, EP_ESTATE, "job has no parameters");
    DeviceGuard g(job->ctx->device);
    cudaError_t e = launch_reset_act(job->precision, static_cast<const DevJob *>(job->dj_dev.p), job->mesh().n_cells,
                                     job->ctx->stream);
    return e == cudaSuccess ? EP_OK : cuda_fail(job->ctx, e, "ep_reset_activation");
}

int ep_step_index(ep_job *job, int64_t *out) {
    if (!job || !out) return EP_EINVAL;
    DeviceGuard g(job->ctx->device);
    long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, job->step_dev.p, sizeof(v), cudaMemcpyDeviceToHost, job->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(job->ctx->stream);
    if (e != cudaSuccess) return cuda_fail(job->ctx, e, "ep_step_index");
    *out = v;
    return EP_OK;
}

int ep_set_step_index(ep_job *job, int64_t n) {
    if (!job || n < 0) return EP_EINVAL;
    DeviceGuard g(job->ctx->device);
    // V lives in buffer (step & 1): move it when the parity changes
    int64_t cur = 0;
    int rc = ep_step_index(job, &cur);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (job->has_params && ((cur ^ n) & 1)) {
        const size_t r = job->precision == EP_FP64_PLAIN ? 8 : 4;
        e = cudaMemcpyAsync(job->dj.V[n & 1], job->dj.V[cur & 1], job->mesh().n_cells * r, cudaMemcpyDeviceToDevice,
                            job->ctx->stream);
        if (e == cudaSuccess && job->gp && job->gp->n > 0)
            e = cudaMemcpyAsync(job->dj.g.V[n & 1], job->dj.g.V[cur & 1], job->gp->n * r, cudaMemcpyDeviceToDevice,
                                job->ctx->stream);
    }
    long long v = n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(job->step_dev.p, &v, sizeof(v), cudaMemcpyHostToDevice, job->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(job->ctx->stream);
    if (e != cudaSuccess) return cuda_fail(job->ctx, e, "ep_set_step_index");
    return restart_ab2(job);
}

int ep_check_finite(ep_job *job) {
    if (!job) return EP_EINVAL;
    if (!job->has_params) return fail(job->ctx, EP_ESTATE, "job has no parameters");
    ep_context *ctx = job->ctx;
    DeviceGuard g(ctx->device);
    DevBuf b;
    int rc = dalloc(ctx, sizeof(unsigned), &b);
    if (rc) return rc;
    unsigned cnt = 0;
    cudaError_t e = cudaMemsetAsync(b.p, 0, sizeof(unsigned), ctx->stream);
    if (e == cudaSuccess)
        e = launch_check_finite(job->precision, static_cast<const DevJob *>(job->dj_dev.p), job->mesh().n_cells,
                                static_cast<unsigned *>(b.p), ctx->stream);
    unsigned werr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, b.p, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&werr, ctx->err_word.p, sizeof(werr), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_check_finite");
    if (werr) {
        *ctx->err_host = werr;
        return fail(ctx, EP_ETIMEOUT, (werr & 1u) ? "a step kernel's wait for its staged copies hit its time limit"
                                                  : "a fused step's wait for its node tiles hit its time limit");
    }
    if (cnt) return fail(ctx, EP_ENONFINITE, std::to_string(cnt) + " non-finite state values");
    return EP_OK;
}

int ep_job_info(const ep_job *job, int64_t *n_cells, int64_t *n_nodes, int64_t *n_interior_faces,
                int64_t *device_bytes, int32_t *index_width, int32_t *node_index_width) {
    if (!job) return EP_EINVAL;
    if (index_width) *index_width = job->sell().idx16 ? 16 : 32;
    if (node_index_width) *node_index_width = job->sell().col16ok ? 16 : 32;
    if (n_cells) *n_cells = job->mesh().n_cells;
    if (n_nodes) *n_nodes = job->mesh().n_nodes;
    if (n_interior_faces) *n_interior_faces = job->mesh().n_interior_faces;
    if (device_bytes) *device_bytes = job->device_bytes;
    return EP_OK;
}

int ep_job_destroy(ep_job *job) {
    if (!job) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_plans_with(ctx, job);
    free_job_arrays(job, &job->prec);
    free_job_arrays(job, &job->topo);
    free_job_arrays(job, &job->gbufs);
    if (job->bido) free_job_arrays(job, &job->bido->bufs);
    dfree(ctx, &job->graph_view);
    dfree(ctx, &job->dj_dev);
    dfree(ctx, &job->step_dev);
    ctx->jobs.erase(job);
    delete job;
    return EP_OK;
}

int ep_plan_inspect(const ep_mesh_desc *desc, const ep_params *params, int64_t *cell_order, int32_t *tet,
                    int32_t *opp, int32_t *nbr, double *wa, double *wb, double *q, int64_t *n2c_ptr,
                    int32_t *n2c, double *nw, double *rho_bound) {
    if (!desc || !params) {
        g_create_error = "ep_plan_inspect: NULL argument";
        return EP_EINVAL;
    }
    try {
        HostMesh m;
        std::string err;
        int rc = build_mesh(desc, &m, &err);
        if (!rc) {
            Coeffs cf;
            if (params->n_sets < 1 || params->n_sets > EP_MAX_PARAM_SETS) {
                err = "ep_plan_inspect: n_sets must be 1..16";
                rc = EP_EINVAL;
            } else {
                rc = build_coeffs(m, params, &cf, &err);
            }
            if (!rc) {
                const int64_t N = m.n_cells;
                auto cp = [](auto *dst, const auto &src) {
                    if (dst) std::copy(src.begin(), src.end(), dst);
                };
                if (cell_order)
                    for (int64_t i = 0; i < N; ++i) cell_order[i] = m.cell_new2old[i];
                cp(tet, m.tet);
                cp(opp, m.opp);
                cp(nbr, m.nbr);
                cp(wa, cf.wa);
                cp(wb, cf.wb);
                cp(q, cf.q);
                cp(n2c_ptr, m.n2c_ptr);
                cp(n2c, m.n2c);
                cp(nw, cf.nw);
                if (rho_bound) *rho_bound = cf.gershgorin;
                return EP_OK;
            }
        }
        g_create_error = err;
        return rc;
    } catch (const std::bad_alloc &) {
        g_create_error = "ep_plan_inspect: out of host memory";
        return EP_ENOMEM;
    }
}

int ep_step_noalloc(ep_job *job, int64_t n_steps) {
    if (!job) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    if (n_steps < 0) return fail(ctx, EP_EINVAL, "ep_step_noalloc: n_steps < 0");
    if (!job->has_params) return fail(ctx, EP_ESTATE, "ep_step_noalloc: the job has no parameters");
    if (job->gp) return fail(ctx, EP_EINVAL, "ep_step_noalloc: jobs with a conduction graph need ep_step");
    if (job->bido) return fail(ctx, EP_EINVAL, "ep_step_noalloc: bidomain jobs need ep_step");
    if (job->params.integrator != EP_INTEGRATOR_FE)
        return fail(ctx, EP_EINVAL, "ep_step_noalloc: AB2 jobs need ep_step");
    if (job->mesh().n_nodes > EP_NOALLOC_MAX_NODES)
        return fail(ctx, EP_EINVAL, "ep_step_noalloc: the mesh has " + std::to_string(job->mesh().n_nodes) +
                                        " nodes; at most " + std::to_string(EP_NOALLOC_MAX_NODES) +
                                        " fit the static node-value array");
    if (job->mesh().n_cells > EP_NOALLOC_MAX_CELLS)
        return fail(ctx, EP_EINVAL, "ep_step_noalloc: the mesh has " + std::to_string(job->mesh().n_cells) +
                                        " cells; at most " + std::to_string(EP_NOALLOC_MAX_CELLS) +
                                        " fit the static tile tables");
    if (*ctx->err_host)
        return fail(ctx, EP_ETIMEOUT, "ep_step_noalloc: an earlier step's bounded wait gave up (ep_clear_error)");
    if (n_steps == 0) return EP_OK;
    DeviceGuard g(ctx->device);
    std::vector<Work> wk;
    const int variant = ctx->cell_variant[job->precision];
    if (is_fused_variant(variant)) append_work(job, 0, 0, &wk);
    cudaError_t e = launch_step_noalloc(job->precision, job->dj, job->node_tiles.data(), int(job->node_tiles.size()),
                                        job->cell_tiles.data(), int(job->cell_tiles.size()), wk.data(),
                                        int(wk.size()), variant, ctx->sm_count,
                                        static_cast<unsigned *>(ctx->err_word.p), n_steps, ctx->stream);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "ep_step_noalloc");
}

int ep_graph_attach(ep_job *job, const ep_graph_desc *desc, const ep_graph_params *params) {
    if (!job || !desc || !params) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    if (!job->has_params) return fail(ctx, EP_ESTATE, "ep_graph_attach: set the job's parameters first");
    DeviceGuard g(ctx->device);
    try {
        std::unique_ptr<GraphPlan> gp(new GraphPlan());
        std::string err;
        int rc = build_graph(job->mesh(), desc, params, &job->params, gp.get(), &err);
        if (rc) return fail(ctx, rc, "ep_graph_attach: " + err);
        job->gp = std::move(gp);
        rc = graph_apply(job);
        if (rc) {
            for (auto &b : job->gbufs) dfree(ctx, &b);
            job->gbufs.clear();
            job->gp.reset();
        }
        return rc;
    } catch (const std::bad_alloc &) {
        return fail(ctx, EP_ENOMEM, "ep_graph_attach: out of host memory");
    }
}

static int graph_io(ep_job *job, int32_t model, int32_t var, double *host, int64_t n, int kind) {
    if (!job) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    if (!job->gp) return fail(ctx, EP_ESTATE, "no conduction graph attached");
    if (!host || n != job->gp->n) return fail(ctx, EP_EINVAL, "buffer length differs from the number of graph nodes");
    if (kind != 2 && (model < 0 || model >= EP_N_MODELS || var < 0 || var >= model_nvar(model)))
        return fail(ctx, EP_EINVAL, "unknown model or variable id");
    if (n == 0) return EP_OK;
    DeviceGuard g(ctx->device);
    DevBuf b;
    int rc = dalloc(ctx, n * sizeof(double), &b);
    if (rc) return rc;
    const DevJob *view = static_cast<const DevJob *>(job->graph_view.p);
    double *buf = static_cast<double *>(b.p);
    cudaError_t e = cudaSuccess;
    if (kind == 1) {
        e = cudaMemcpyAsync(buf, host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_scatter(job->precision, view, job->gperm_dev, n, model, var, buf, ctx->stream);
    } else {
        e = kind == 0 ? launch_gather(job->precision, view, job->gperm_dev, n, model, var, buf, ctx->stream)
                      : launch_gather_act(job->precision, view, job->gperm_dev, n, buf, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, "graph state transfer");
}

int ep_graph_read_state(ep_job *job, int32_t model, int32_t var, double *host_out, int64_t n) {
    return graph_io(job, model, var, host_out, n, 0);
}

int ep_graph_write_state(ep_job *job, int32_t model, int32_t var, const double *host_in, int64_t n) {
    return graph_io(job, model, var, const_cast<double *>(host_in), n, 1);
}

int ep_graph_activation_times(ep_job *job, double *host_out, int64_t n) {
    return graph_io(job, 0, 0, host_out, n, 2);
}

int ep_graph_info(const ep_job *job, int64_t *n_nodes, int32_t *substeps, int64_t *n_junctions) {
    if (!job) return EP_EINVAL;
    if (n_nodes) *n_nodes = job->gp ? job->gp->n : 0;
    if (substeps) *substeps = job->gp ? job->gp->substeps : 0;
    if (n_junctions) *n_junctions = job->gp ? int64_t(job->gp->jnode.size()) : 0;
    return EP_OK;
}

int ep_bidomain_enable(ep_job *job, const double *De_l, const double *De_t, int32_t n_sets,
                       const ep_bidomain_solver *solver) {
    if (!job) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    if (!job->has_params) return fail(ctx, EP_ESTATE, "ep_bidomain_enable: job has no parameters");
    for (uint8_t k : job->mesh().kind)
        if (k) return fail(ctx, EP_EINVAL, "ep_bidomain_enable: the Purkinje shell is a monodomain medium");
    if (!De_l || !De_t || n_sets != job->params.n_sets)
        return fail(ctx, EP_EINVAL, "ep_bidomain_enable: need one extracellular (D_l, D_t) per parameter set");
    ep_bidomain_solver sv;
    if (solver) {
        sv = *solver;
    } else {
        const bool plain = job->precision == EP_FP64_PLAIN;
        sv = ep_bidomain_solver{plain ? 1e-11 : 1e-5, plain ? 1e-11 : 1e-3, 12, 0, 2000, 0.0};
    }
    if (!(sv.barrier_limit_s > 0.0)) sv.barrier_limit_s = 2.0;
    if (sv.barrier_limit_s > 60.0)
        return fail(ctx, EP_EINVAL, "ep_bidomain_enable: barrier_limit_s above 60 s");
    if (!(sv.tol > 0.0) || !(sv.atol >= 0.0) || sv.restart < 1 || sv.restart > kBidoMaxRestart || sv.max_iter < 1 ||
        (sv.reorth != 0 && sv.reorth != 1))
        return fail(ctx, EP_EINVAL, "ep_bidomain_enable: tol > 0, atol >= 0, restart 1..30, reorth 0/1, max_iter >= 1");
    for (int k = 0; k < n_sets; ++k)
        if (!(De_l[k] >= 0.0) || !(De_t[k] >= 0.0))
            return fail(ctx, EP_EINVAL, "ep_bidomain_enable: negative extracellular diffusivity");
    DeviceGuard g(ctx->device);
    try {
        if (!job->bido) job->bido.reset(new BidoHost());
        BidoHost &B = *job->bido;
        B.De_l.assign(De_l, De_l + n_sets);
        B.De_t.assign(De_t, De_t + n_sets);
        B.tol = sv.tol;
        B.atol = sv.atol;
        B.restart = sv.restart;
        B.reorth = sv.reorth;
        B.max_iter = sv.max_iter;
        B.barrier_limit_s = sv.barrier_limit_s;
        int rc = bido_apply(job);
        if (rc) bido_drop(job);
        return rc;
    } catch (const std::bad_alloc &) {
        bido_drop(job);
        return fail(ctx, EP_ENOMEM, "ep_bidomain_enable: out of host memory");
    }
}

int ep_bidomain_disable(ep_job *job) {
    if (!job) return EP_EINVAL;
    DeviceGuard g(job->ctx->device);
    bido_drop(job);
    return EP_OK;
}

static int transfer_ve(ep_job *job, double *host, int64_t n, bool write) {
    int rc = check_io(job, n, host);
    if (rc) return rc;
    ep_context *ctx = job->ctx;
    if (!job->bido) return fail(ctx, EP_ESTATE, "job is not bidomain (ep_bidomain_enable)");
    DeviceGuard g(ctx->device);
    DevBuf b;
    if ((rc = dalloc(ctx, n * sizeof(double), &b))) return rc;
    double *buf = static_cast<double *>(b.p);
    cudaError_t e;
    if (write) {
        BidoArgs a = job->bido->args;
        a.mode = 1;   // refresh L_i(v_e) for the next step
        e = cudaMemcpyAsync(buf, host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_field_scatter(job->precision, buf, job->perm_dev, n, a.ve, ctx->stream);
        // a restored v_e ends the record of a solve whose barrier gave up
        if (e == cudaSuccess)
            e = cudaMemsetAsync(reinterpret_cast<char *>(a.stats) + offsetof(BidoStats, timeout), 0, sizeof(int),
                                ctx->stream);
        if (e == cudaSuccess) e = launch_bido(job->precision, a, job->dj, job->bido->grid, ctx->stream);
    } else {
        e = launch_field_gather(job->precision, job->bido->args.ve, job->perm_dev, n, buf, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, &b);
    return e == cudaSuccess ? EP_OK : cuda_fail(ctx, e, write ? "ep_bidomain_write_ve" : "ep_bidomain_read_ve");
}

int ep_bidomain_read_ve(ep_job *job, double *host_out, int64_t n) {
    try {
        return transfer_ve(job, host_out, n, false);
    } catch (const std::bad_alloc &) {
        return fail(job->ctx, EP_ENOMEM, "ep_bidomain_read_ve: out of host memory");
    }
}

int ep_bidomain_write_ve(ep_job *job, const double *host_in, int64_t n) {
    try {
        return transfer_ve(job, const_cast<double *>(host_in), n, true);
    } catch (const std::bad_alloc &) {
        return fail(job->ctx, EP_ENOMEM, "ep_bidomain_write_ve: out of host memory");
    }
}

int ep_bidomain_stats(ep_job *job, ep_bidomain_stats_t *out) {
    if (!job || !out) return EP_EINVAL;
    ep_context *ctx = job->ctx;
    if (!job->bido) return fail(ctx, EP_ESTATE, "job is not bidomain (ep_bidomain_enable)");
    DeviceGuard g(ctx->device);
    BidoStats st{};
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&st, job->bido->args.stats, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ep_bidomain_stats");
    *out = ep_bidomain_stats_t{};
    out->last_iters = st.last_iters;
    out->total_iters = st.total_iters;
    out->solves = st.solves;
    out->last_res = st.last_res;
    out->last_bnorm = st.last_bnorm;
    out->alg_bytes = st.alg_bytes;
    for (int k = 0; k < 5; ++k) out->phase_ms[k] = st.phase_ms[k];
    out->failed = st.failed;
    out->timeout = st.timeout;
    if (st.timeout) return fail(ctx, EP_ETIMEOUT, "bidomain solve: a grid barrier wait hit its time limit");
    return EP_OK;
}

}  // extern "C"
