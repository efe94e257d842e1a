// Device kernels of the monodomain finite-volume step (Sec. 3.2).
//
// One step of every resident job is two launches:
//   node_kernel  S1: v_n = sum_k w_nk V_k over the cells around each node
//                (inverse-distance weights, sliced-ELL table, coalesced);
//   cell_kernel  S2 + S3 + the cell model, fused: the diffusion term of
//                Eqs. 7-8 from eight node values and four neighbour
//                potentials with folded FP64-derived coefficients, then the
//                cell model (Rush-Larsen / forward Euler at (V^n, s^n)),
//                the stimulus of Eq. 4, V^{n+1} and the activation time.
// Both kernels are persistent (grid-stride over tiles of one job and one
// model) and serve every job of a launch group in one launch. The last block
// of the cell launch advances the jobs' step counters, which select the V
// buffer (double-buffered by step parity) and the time t^n = n dt. This file
// holds the kernels that read the jobs' descriptors from the job table in
// global memory, and the launch dispatch; kernels_tab.cu the FP32 kernels
// whose descriptors are a kernel parameter, kernels_f64.cu the FP64 cell
// kernel shapes, cellstep.cuh the device code they share.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "cellstep.cuh"

namespace ep {

// F: the form of the batch's node -> cell entries (0 all 32-bit, 1 all
// 16-bit, 2 mixed), so that a uniform batch compiles one form only.
template <class R, int F>
__global__ void __launch_bounds__(kNodeThreads) node_kernel(const DevJob *__restrict__ jobs,
                                                            const Tile *__restrict__ tiles, int n_tiles) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const DevJob &J = jobs[tl.job];
        const int i = threadIdx.x;
        if (i >= tl.count) continue;
        const long long node = (long long)tl.start + i;
        const long long n = *J.step;
        const R *__restrict__ V = static_cast<const R *>(J.V[n & 1]);
        static_cast<R *>(J.vn)[node] = node_value<R, 6, F>(J, V, node);
    }
}

template <class R>
static void launch_node_kernel(const StepLaunch &L, cudaStream_t s) {
    if constexpr (std::is_same<R, float>::value) {
        if (tab_eligible(L)) {
            launch_node_tab(L, s);
            return;
        }
    }
    auto *k = L.node_form == 0 ? node_kernel<R, 0> : (L.node_form == 1 ? node_kernel<R, 1> : node_kernel<R, 2>);
    k<<<L.node_grid, kNodeThreads, 0, s>>>(L.jobs, L.node_tiles, L.n_node_tiles);
}

// Conduction graph, part 1 (Sec. 3.2 / 3.3): the reaction of every graph node
// at (V^n, s^n) -- cell model, stimulus protocols, antidromic triggered
// stimulus and resistive junction current -- frozen for the step's substeps.
template <class R>
__global__ void __launch_bounds__(kGraphThreads) graph_ionic_kernel(const DevJob *__restrict__ jobs,
                                                                    const Tile *__restrict__ tiles, int n_tiles) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const DevJob &J = jobs[tl.job];
        const DevGraph &G = J.g;
        for (int i = threadIdx.x; i < tl.count; i += blockDim.x) {
            const long long node = (long long)tl.start + i;
            const long long n = *J.step;
            const double tn = double(n) * J.dt;
            const R Vg = static_cast<const R *>(G.V[n & 1])[node];
            const R *V3 = static_cast<const R *>(J.V[n & 1]);
            const unsigned mask = G.smask[node];
            R is = mask ? stimulus<R>(J, mask, n) : R(0);
            R ix = R(0);
            for (int k = G.node_junc_ptr[node]; k < G.node_junc_ptr[node + 1]; ++k) {
                const int j = G.node_junc[k];
                if (G.jmode[j] == EP_PMJ_RESISTIVE) ix += pick<R>(G.g_graph, G.g_graph_f) * (Vg - V3[G.jcell[j]]);
                else if (G.jmode[j] == EP_PMJ_TRIGGERED && G.two_way && window_on(G.t_cell[j], G.delay_anti, G.duration, tn))
                    is += pick<R>(G.amplitude, G.amplitude_f);
            }
            const DevParams &P = J.params[G.pset[node]];
            const R dt = pick<R>(J.dt, J.dt_f);
            const DevRegion &rg = G.reg[tl.model];
            const long long li = node - rg.off;
            R iion;
            const CellIO<R> io = region_io<R>(rg, li);
            if (tl.model == EP_TP06) iion = tt_step<R, false>(io, P, Vg, dt, is);
            else if (tl.model == EP_STEWART) iion = tt_step<R, true>(io, P, Vg, dt, is);
            else iion = crn_step<R>(io, P, Vg, dt);
            static_cast<R *>(G.itot)[node] = iion + is + ix;
        }
    }
}

// Conduction graph, part 2: diffusion substep s of each job's k substeps of
// h = dt / k (a job with fewer substeps than the batch's largest copies its
// values through). The last substep writes V^{n+1}, the activation times and
// the graph-side junction crossings.
template <class R>
__global__ void __launch_bounds__(kGraphThreads) graph_diffuse_kernel(const DevJob *__restrict__ jobs,
                                                                      const Tile *__restrict__ tiles, int n_tiles,
                                                                      int s, int last) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const DevJob &J = jobs[tl.job];
        const DevGraph &G = J.g;
        const long long n = *J.step;
        const R *Win = static_cast<const R *>(s == 0 ? G.V[n & 1] : G.W[s & 1]);
        const R *cf = static_cast<const R *>(G.coef);
        for (int i = threadIdx.x; i < tl.count; i += blockDim.x) {
            const long long node = (long long)tl.start + i;
            const R w = Win[node];
            R out = w;
            if (s < G.substeps) {
                R lap = R(0);
                for (int e = G.row[node]; e < G.row[node + 1]; ++e) lap += cf[e] * (Win[G.col[e]] - w);
                out = w + pick<R>(G.h, G.h_f) * (lap - static_cast<const R *>(G.itot)[node]);
            }
            if (!last) {
                static_cast<R *>(G.W[(s + 1) & 1])[node] = out;
                continue;
            }
            static_cast<R *>(G.V[(n & 1) ^ 1])[node] = out;
            const R v0 = static_cast<const R *>(G.V[n & 1])[node];
            const R th = pick<R>(J.threshold, J.threshold_f);
            if (v0 < th && out >= th) {
                R *act = static_cast<R *>(G.act);
                if (isinf(act[node])) act[node] = R(double(n) * J.dt) + pick<R>(J.dt, J.dt_f) * (th - v0) / (out - v0);
            }
            const double gth = G.threshold;
            if (double(v0) < gth && double(out) >= gth)
                for (int k = G.node_junc_ptr[node]; k < G.node_junc_ptr[node + 1]; ++k) {
                    const int j = G.node_junc[k];
                    if (G.jmode[j] == EP_PMJ_TRIGGERED)
                        G.t_graph[j] = double(n) * J.dt + J.dt * (gth - double(v0)) / (double(out) - double(v0));
                }
        }
    }
}

// Conduction graph, part 2, all substeps in one launch: each block takes a
// graph tile and its nodes' neighbourhood up to the job's substep count in
// hops (host tables), runs every substep in shared memory -- the values of
// the tile's own nodes stay exact, since an error at the rim of the
// neighbourhood travels one hop per substep -- and writes the tile's
// V^{n+1}, activation times and junction crossings. Per node the arithmetic
// and its order are those of graph_diffuse_kernel, so the results are the
// same bit for bit, with one launch per step instead of one per substep.
template <class R>
__global__ void __launch_bounds__(kGraphThreads) graph_substeps_kernel(const DevJob *__restrict__ jobs,
                                                                       const Tile *__restrict__ tiles, int n_tiles,
                                                                       int n_sub, int lmax) {
    extern __shared__ __align__(16) unsigned char gsm[];
    R *const wa = reinterpret_cast<R *>(gsm);
    R *const wb = wa + lmax;
    R *const it = wb + lmax;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const DevJob &J = jobs[tl.job];
        const DevGraph &G = J.g;
        const long long n = *J.step;
        const int s0 = G.lt_ptr[tl.model], L = G.lt_ptr[tl.model + 1] - s0;
        const R *Vin = static_cast<const R *>(G.V[n & 1]);
        const R *itot = static_cast<const R *>(G.itot);
        const R *cf = static_cast<const R *>(G.coef);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const int u = G.lslot[s0 + i].x;
            wa[i] = Vin[u];
            it[i] = itot[u];
        }
        __syncthreads();
        R *cur = wa, *nxt = wb;
        for (int s = 0; s < n_sub; ++s) {
            for (int i = threadIdx.x; i < L; i += blockDim.x) {
                const R w = cur[i];
                R out = w;
                if (s < G.substeps) {
                    const int2 sl = G.lslot[s0 + i];
                    R lap = R(0);
                    for (int e = G.row[sl.x], k = sl.y; e < G.row[sl.x + 1]; ++e, ++k) {
                        const int j = G.lcol[k];
                        lap += cf[e] * ((j >= 0 ? cur[j] : w) - w);   // -1: beyond the rim, never read by the tile
                    }
                    out = w + pick<R>(G.h, G.h_f) * (lap - it[i]);
                }
                nxt[i] = out;
            }
            __syncthreads();
            R *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        for (int i = threadIdx.x; i < tl.count; i += blockDim.x) {
            const long long node = (long long)tl.start + i;
            const R out = cur[i];
            static_cast<R *>(G.V[(n & 1) ^ 1])[node] = out;
            const R v0 = Vin[node];
            const R th = pick<R>(J.threshold, J.threshold_f);
            if (v0 < th && out >= th) {
                R *act = static_cast<R *>(G.act);
                if (isinf(act[node])) act[node] = R(double(n) * J.dt) + pick<R>(J.dt, J.dt_f) * (th - v0) / (out - v0);
            }
            const double gth = G.threshold;
            if (double(v0) < gth && double(out) >= gth)
                for (int k = G.node_junc_ptr[node]; k < G.node_junc_ptr[node + 1]; ++k) {
                    const int j = G.node_junc[k];
                    if (G.jmode[j] == EP_PMJ_TRIGGERED)
                        G.t_graph[j] = double(n) * J.dt + J.dt * (gth - double(v0)) / (double(out) - double(v0));
                }
        }
        __syncthreads();   // the shared arrays are refilled for the next tile
    }
}

// ---------------------------------------------------------------------------
// Fused step: the node values (S1) and the cell update of every job in ONE
// persistent launch. The launch works through a list of node tiles and cell
// tiles (Work), claimed in order from a device counter by each warp. A cell tile of a job
// needs the values of a bounded range of that job's node tiles (the gather
// indices of an RCM-numbered mesh are local), and the host orders the list
// so that those node tiles come first, queued kFusedLookahead cell tiles
// ahead. Node tiles are counted complete per chunk of kFusedChunk tiles: a
// block that finishes a node tile adds one to its chunk's counter with
// release semantics, so after g fused launches a chunk of k tiles holds
// g k, and in launch g (the job's launch counter, read at the start) the
// chunk is complete once it holds (g + 1) k. A warp that claims a cell tile
// polls the chunks of its range with relaxed loads (one lane each), then
// acquires with one fence per lane, then reads the node values. Every wait
// ends (see the kernel), and is bounded all the same. The V^n a node tile reads is read again soon after
// by the cell tiles of the same region, from L2. The last block to finish
// advances each job's step and launch counters and re-arms the work counter.
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long kFusedWaitLimitNs = 1000000000ull;   // 1 s

template <class R, int T, int MINB, bool XD, bool AB2>
__global__ void __launch_bounds__(T, MINB)
    fused_kernel(const DevJob *__restrict__ jobs, const Tile *__restrict__ node_tiles,
                 const Tile *__restrict__ cell_tiles, const Work *__restrict__ work, int n_work, unsigned *head,
                 unsigned *done, int n_jobs, unsigned *err) {
    // Every warp claims and works through whole items on its own (no block
    // barrier per item), and claims its next item before working on the
    // current one, so the claim's latency overlaps the work. A warp's items
    // are in increasing list order, so the oldest claimed, unfinished item is
    // always being worked on and its wait (if a cell tile) is on finished
    // node tiles: every wait ends.
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int next = 0;
    if (lane == 0) next = int(atomicAdd(head, 1u));
    next = __shfl_sync(full, next, 0);
    while (next < n_work) {
        const int it = next;
        if (lane == 0) next = int(atomicAdd(head, 1u));
        const Work wk = work[it];
        if (wk.tile < 0) {
            const Tile tl = node_tiles[-1 - wk.tile];
            const DevJob &J = jobs[tl.job];
            const long long n = *J.step;
            const R *__restrict__ V = static_cast<const R *>(J.V[n & 1]);
            R *vn = static_cast<R *>(J.vn);
            // two nodes per lane at a time, their gathers in flight together
            for (int i = lane; i < tl.count; i += 64) {
                const long long a = (long long)tl.start + i, b = a + 32;
                const bool hb = i + 32 < tl.count;
                const R va = node_value<R>(J, V, a);
                const R vb = hb ? node_value<R>(J, V, b) : R(0);
                vn[a] = va;
                if (hb) vn[b] = vb;
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                red_release_add(J.ntflag + ((tl.start / kNodeThreads) / kFusedChunk), 1u);
            }
        } else {
            const Tile tl = cell_tiles[wk.tile];
            const DevJob &J = jobs[tl.job];
            const unsigned tag = *J.gen + 1u;
            const int n_nt = int((J.n_nodes + kNodeThreads - 1) / kNodeThreads);
            const int c0 = wk.dep_lo / kFusedChunk, c1 = wk.dep_hi / kFusedChunk;
            bool polled = false;
            for (int ch = c0 + lane; ch <= c1; ch += 32) {
                const unsigned want = tag * unsigned(min(kFusedChunk, n_nt - ch * kFusedChunk));
                polled = true;
                if (ld_relaxed(J.ntflag + ch) >= want) continue;
                const unsigned long long t0 = global_timer_ns();
                while (ld_relaxed(J.ntflag + ch) < want) {
                    if (global_timer_ns() - t0 > kFusedWaitLimitNs) {
                        atomicOr(err, 2u);   // reported by ep_step / ep_check_finite; the tile goes on
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (polled) fence_acq_rel_gpu();   // acquire what the chunks' releases published
            __syncwarp();
            for (int i = lane; i < tl.count; i += 32)
                cell_update<R, XD, AB2, true>(J, tl.model, (long long)tl.start + i);
        }
        next = __shfl_sync(full, next, 0);
    }
    // Every warp has read the counters; the last block to finish advances them.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            for (int j = 0; j < n_jobs; ++j) {
                *jobs[j].step += 1;
                *jobs[j].gen += 1u;
            }
            *head = 0u;
            *done = 0u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Staged cell kernel (FP32, forward Euler). The streamed inputs of a tile --
// its cells' vertex / opposite-vertex / neighbour indices, folded
// coefficients, state arrays, accumulators, V and the stimulus / parameter
// bytes, all contiguous runs -- are brought into shared memory by bulk
// asynchronous copies (cp.async.bulk, the TMA engine) issued by one thread,
// double-buffered: while the block computes tile k from one stage, the copies
// of tile k+1 land in the other, so the cell updates do not wait on HBM
// latency for their own data. Gathers (node values, neighbour potentials)
// still go through L2. Arithmetic and results are those of cell_kernel.
namespace staged {

constexpr int kCells = kCellThreads;   // one tile: up to 256 consecutive cells of one model
constexpr int kMaxR = 16, kMaxA = 4;   // state arrays of the largest model

// STATE: the tile's state arrays and accumulators are staged too (the full
// stage, two blocks per SM), or only its indices, coefficients, V and bytes
// (a third of the size, three blocks per SM), the state being read directly.
template <bool STATE> struct StageState;
template <> struct StageState<true> {
    float r[kMaxR][kCells];
    double a[kMaxA][kCells];
};
template <> struct StageState<false> {};
template <bool STATE>
struct Stage : StageState<STATE> {
    int4 na[kCells], nb[kCells], nc[kCells];
    float4 wa[kCells], wb[kCells], q[kCells];
    float V[kCells];
    uint8_t smask[kCells], pset[kCells];
};
template <bool STATE>
struct Shared {
    Stage<STATE> st[2];
    unsigned long long bar[2];
    int flags[2];   // bit 0: V staged, bit 1: stimulus / parameter bytes staged
};
template <bool STATE> constexpr size_t smem_bytes() { return sizeof(Shared<STATE>); }
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned s_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(unsigned long long *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, unsigned long long *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(s_addr(dst)), "l"(src), "r"(bytes), "r"(s_addr(b))
                 : "memory");
}
// Bounded wait on a stage's barrier; false (and the error flag set) past the limit.
__device__ __forceinline__ bool bar_wait(unsigned long long *b, unsigned parity, unsigned *err) {
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (!bar_try(b, parity)) {
        if (now_ns() - t0 > kWaitLimitNs) {
            atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ unsigned r16(unsigned b) { return (b + 15u) & ~15u; }

// Issue the copies of tile tl into stage s (one thread). The region arrays are
// padded to a multiple of 64 cells and a tile starts at a multiple of 256
// cells inside its region, so rounding their sizes up to 16 bytes stays in
// bounds; V and the byte arrays are staged only when their runs are aligned.
template <bool STATE>
__device__ void issue(const DevJob &J, const Tile &tl, Stage<STATE> &S, unsigned long long *bar, int *flags, int nr,
                      int nA) {
    const long long c0 = tl.start;
    const unsigned cnt = unsigned(tl.count);
    const DevRegion &rg = J.reg[tl.model];
    const long long i0 = c0 - rg.off;
    const long long step = *J.step;
    const float *V = static_cast<const float *>(J.V[step & 1]);
    const bool sv = (c0 % 4 == 0) && (cnt % 4 == 0);
    const bool sb = (c0 % 16 == 0) && (cnt % 16 == 0);
    *flags = (sv ? 1 : 0) | (sb ? 2 : 0);
    unsigned total = 6u * cnt * 16u;
    if constexpr (STATE) total += unsigned(nr) * r16(cnt * 4u) + unsigned(nA) * r16(cnt * 8u);
    if (sv) total += cnt * 4u;
    if (sb) total += 2u * cnt;
    bar_expect(bar, total);
    bulk_copy(S.na, J.nodes_a + c0, cnt * 16u, bar);
    bulk_copy(S.nb, J.nodes_b + c0, cnt * 16u, bar);
    bulk_copy(S.nc, J.nbr + c0, cnt * 16u, bar);
    bulk_copy(S.wa, static_cast<const float4 *>(J.wa) + c0, cnt * 16u, bar);
    bulk_copy(S.wb, static_cast<const float4 *>(J.wb) + c0, cnt * 16u, bar);
    bulk_copy(S.q, static_cast<const float4 *>(J.q) + c0, cnt * 16u, bar);
    if constexpr (STATE) {
        const float *r = static_cast<const float *>(rg.r) + i0;
        for (int v = 0; v < nr; ++v) bulk_copy(S.r[v], r + v * rg.stride, r16(cnt * 4u), bar);
        const double *a = rg.a + i0;
        for (int k = 0; k < nA; ++k) bulk_copy(S.a[k], a + k * rg.stride, r16(cnt * 8u), bar);
    }
    if (sv) bulk_copy(S.V, V + c0, cnt * 4u, bar);
    if (sb) {
        bulk_copy(S.smask, J.smask + c0, cnt, bar);
        bulk_copy(S.pset, J.pset + c0, cnt, bar);
    }
}

}  // namespace staged

template <bool XD, bool STATE>
__global__ void __launch_bounds__(kCellThreads, STATE ? 2 : 3)
    cell_kernel_staged(const DevJob *__restrict__ jobs, const Tile *__restrict__ tiles, int n_tiles, unsigned *done,
                       int n_jobs, unsigned *err) {
    using namespace staged;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Shared<STATE> &sh = *reinterpret_cast<Shared<STATE> *>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) {
        bar_init(&sh.bar[0]);
        bar_init(&sh.bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int k = 0;
    int t = blockIdx.x;
    if (tid == 0 && t < n_tiles) {
        const Tile tl = tiles[t];
        issue(jobs[tl.job], tl, sh.st[0], &sh.bar[0], &sh.flags[0], model_nr(tl.model), model_na(tl.model));
    }
    bool ok = true;
    for (; t < n_tiles; t += gridDim.x, ++k) {
        const int s = k & 1;
        // prefetch the next tile into the other stage (its readers finished at the last barrier)
        const int tn = t + gridDim.x;
        if (tid == 0 && tn < n_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const Tile tl = tiles[tn];
            issue(jobs[tl.job], tl, sh.st[s ^ 1], &sh.bar[s ^ 1], &sh.flags[s ^ 1], model_nr(tl.model),
                  model_na(tl.model));
        }
        // every thread waits (acquiring the copied data); the block then agrees on the outcome
        const bool arrived = bar_wait(&sh.bar[s], unsigned((k >> 1) & 1), err);
        if (!__syncthreads_and(arrived)) {
            ok = false;
            break;
        }
        const Tile tl = tiles[t];
        const DevJob &J = jobs[tl.job];
        const Stage<STATE> &S = sh.st[s];
        const int fl = sh.flags[s];
        if (tid < tl.count) {
            const long long c = (long long)tl.start + tid;
            const long long n = *J.step;
            const float *V = static_cast<const float *>(J.V[n & 1]);
            const DevRegion &rg = J.reg[tl.model];
            const long long li = c - rg.off;
            CellIO<float> io = region_io<float>(rg, li);
            if constexpr (STATE) {
                io.xi = &S.r[0][tid];
                io.ai = &S.a[0][tid];
                io.si = kCells;
            }
            CellSrc<float> src{S.na[tid], S.nb[tid], S.nc[tid], S.wa + tid, S.wb + tid, S.q + tid,
                               (fl & 1) ? S.V + tid : V + c, (fl & 2) ? S.smask + tid : J.smask + c,
                               (fl & 2) ? S.pset + tid : J.pset + c, io};
            cell_update_from<float, XD, false>(J, tl.model, c, n, V, src);
        }
        __syncthreads();
    }
    if (!ok && tid == 0) {
        // a copy did not complete in time: wait (bounded) for the copies still in flight --
        // tile k's and, if issued, tile k+1's -- before the block's shared memory is released
        bar_wait(&sh.bar[k & 1], unsigned((k >> 1) & 1), err);
        if (t + int(gridDim.x) < n_tiles) bar_wait(&sh.bar[(k + 1) & 1], unsigned(((k + 1) >> 1) & 1), err);
    }
    // Every block has read the step counters; the last one to finish advances them.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            for (int j = 0; j < n_jobs; ++j) *jobs[j].step += 1;
            *done = 0u;
            __threadfence();
        }
    }
}

template <class R>
__global__ void init_kernel(const DevJob *__restrict__ job, long long n_cells) {
    const DevJob &J = *job;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        int model = 0;
        while (model < EP_N_MODELS - 1 && c >= J.reg[model].off + J.reg[model].n) ++model;
        const DevRegion &rg = J.reg[model];
        R v;
        if (model == EP_TP06) tt_init<R, false>(rg, c - rg.off, &v);
        else if (model == EP_STEWART) tt_init<R, true>(rg, c - rg.off, &v);
        else crn_init<R>(rg, c - rg.off, &v);
        static_cast<R *>(J.V[0])[c] = v;
        static_cast<R *>(J.V[1])[c] = v;
        static_cast<R *>(J.act)[c] = R(INFINITY);
    }
}

struct DevVarLoc {
    int kind, slot;
};

// out / in are in the caller's cell order: internal cell c is caller cell perm[c].
// H: the caller's element type (double; or float for the variables an FP32
// job stores in FP32, exactly).
template <class R, class H = double>
__global__ void gather_kernel(const DevJob *__restrict__ job, const int *__restrict__ perm, long long n_cells,
                              int model, DevVarLoc loc, H *buf, int write) {
    const DevJob &J = *job;
    const long long n = *J.step;
    R *V = static_cast<R *>(J.V[n & 1]);
    const DevRegion &rg = J.reg[model];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        H &x = buf[perm[c]];
        if (loc.kind == kVarV) {
            if (write) V[c] = R(x);
            else x = H(V[c]);
            continue;
        }
        if (c < rg.off || c >= rg.off + rg.n) {
            if (!write) x = H(NAN);
            continue;
        }
        const long long i = c - rg.off;
        if (loc.kind == kVarR) {
            R *p = static_cast<R *>(rg.r) + loc.slot * rg.stride + i;
            if (write) *p = R(x);
            else x = H(*p);
        } else {
            double *p = rg.a + loc.slot * rg.stride + i;
            if (write) Accum<R>::init(p, double(x));
            else x = H(Accum<R>::read(p));
        }
    }
}

template <class R, class H = double>
__global__ void act_kernel(const DevJob *__restrict__ job, const int *__restrict__ perm, long long n_cells,
                           H *out) {
    R *act = static_cast<R *>(job->act);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        if (out) out[perm[c]] = H(act[c]);
        else act[c] = R(INFINITY);
    }
}

template <class R>
__global__ void finite_kernel(const DevJob *__restrict__ job, long long n_cells, unsigned *count) {
    const DevJob &J = *job;
    const long long n = *J.step;
    const R *V = static_cast<const R *>(J.V[n & 1]);
    unsigned bad = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        if (!isfinite(V[c])) ++bad;
        int model = 0;
        while (model < EP_N_MODELS - 1 && c >= J.reg[model].off + J.reg[model].n) ++model;
        const DevRegion &rg = J.reg[model];
        const long long i = c - rg.off;
        for (int k = 0; k < model_nr(model); ++k)
            if (!isfinite(static_cast<const R *>(rg.r)[k * rg.stride + i])) ++bad;
        for (int k = 0; k < model_na(model); ++k)
            if (!isfinite(Accum<R>::read(rg.a + k * rg.stride + i))) ++bad;
    }
    if (bad) atomicAdd(count, bad);
}

static int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    return int(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

template <class R>
static cudaError_t graph_impl(const StepLaunch &L, cudaStream_t s) {
    if (L.n_graph_tiles > 0) {
        graph_ionic_kernel<R><<<L.graph_grid, kGraphThreads, 0, s>>>(L.jobs, L.graph_tiles, L.n_graph_tiles);
        if (L.graph_local && 3 * size_t(L.graph_lmax) * sizeof(R) <= kGraphLocalMaxBytes) {
            graph_substeps_kernel<R><<<L.graph_grid, kGraphThreads, 3 * size_t(L.graph_lmax) * sizeof(R), s>>>(
                L.jobs, L.graph_sub_tiles, L.n_graph_tiles, L.graph_substeps, L.graph_lmax);
        } else {
            for (int k = 0; k < L.graph_substeps; ++k)
                graph_diffuse_kernel<R><<<L.graph_grid, kGraphThreads, 0, s>>>(L.jobs, L.graph_tiles,
                                                                               L.n_graph_tiles, k,
                                                                               k == L.graph_substeps - 1);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_graph(int precision, const StepLaunch &L, cudaStream_t s) {
    return precision == EP_FP64_PLAIN ? graph_impl<double>(L, s) : graph_impl<float>(L, s);
}

template <class R>
static cudaError_t step_impl(const StepLaunch &L, cudaStream_t s) {
    // the conduction graphs read no node values: with the fused variants they run first
    if (!is_fused_variant(L.cell_variant)) launch_node_kernel<R>(L, s);
    graph_impl<R>(L, s);
    return launch_cell(sizeof(R) == 8 ? EP_FP64_PLAIN : EP_FP32_MIXED, L, s);
}

cudaError_t launch_step(int precision, const StepLaunch &L, cudaStream_t s) {
    return precision == EP_FP64_PLAIN ? step_impl<double>(L, s) : step_impl<float>(L, s);
}

cudaError_t launch_init(int precision, const DevJob *job, long long n_cells, cudaStream_t s) {
    if (precision == EP_FP64_PLAIN) init_kernel<double><<<grid_for(n_cells, 256), 256, 0, s>>>(job, n_cells);
    else init_kernel<float><<<grid_for(n_cells, 256), 256, 0, s>>>(job, n_cells);
    return cudaGetLastError();
}

static cudaError_t gather_impl(int precision, const DevJob *job, const int *perm, long long n_cells, int model,
                               int var, double *buf, int write, cudaStream_t s) {
    const VarLoc &v = model_vars(model)[var];
    DevVarLoc loc{v.kind, v.slot};
    if (precision == EP_FP64_PLAIN)
        gather_kernel<double><<<grid_for(n_cells, 256), 256, 0, s>>>(job, perm, n_cells, model, loc, buf, write);
    else
        gather_kernel<float><<<grid_for(n_cells, 256), 256, 0, s>>>(job, perm, n_cells, model, loc, buf, write);
    return cudaGetLastError();
}

cudaError_t launch_gather(int precision, const DevJob *job, const int *perm, long long n_cells, int model, int var,
                          double *out, cudaStream_t s) {
    return gather_impl(precision, job, perm, n_cells, model, var, out, 0, s);
}

cudaError_t launch_scatter(int precision, const DevJob *job, const int *perm, long long n_cells, int model, int var,
                           const double *in, cudaStream_t s) {
    return gather_impl(precision, job, perm, n_cells, model, var, const_cast<double *>(in), 1, s);
}

cudaError_t launch_gather_act(int precision, const DevJob *job, const int *perm, long long n_cells, double *out,
                              cudaStream_t s) {
    if (precision == EP_FP64_PLAIN)
        act_kernel<double><<<grid_for(n_cells, 256), 256, 0, s>>>(job, perm, n_cells, out);
    else
        act_kernel<float><<<grid_for(n_cells, 256), 256, 0, s>>>(job, perm, n_cells, out);
    return cudaGetLastError();
}

cudaError_t launch_transfer_f32(const DevJob *job, const int *perm, long long n_cells, int model, int var,
                                float *buf, int write, cudaStream_t s) {
    const VarLoc &v = model_vars(model)[var];
    gather_kernel<float, float><<<grid_for(n_cells, 256), 256, 0, s>>>(job, perm, n_cells, model,
                                                                       DevVarLoc{v.kind, v.slot}, buf, write);
    return cudaGetLastError();
}

cudaError_t launch_gather_act_f32(const DevJob *job, const int *perm, long long n_cells, float *out, cudaStream_t s) {
    act_kernel<float, float><<<grid_for(n_cells, 256), 256, 0, s>>>(job, perm, n_cells, out);
    return cudaGetLastError();
}

cudaError_t launch_reset_act(int precision, const DevJob *job, long long n_cells, cudaStream_t s) {
    return launch_gather_act(precision, job, nullptr, n_cells, nullptr, s);
}

cudaError_t launch_node(int precision, const StepLaunch &L, cudaStream_t s) {
    if (is_fused_variant(L.cell_variant)) return cudaSuccess;   // the fused launch computes the node values
    if (precision == EP_FP64_PLAIN) launch_node_kernel<double>(L, s);
    else launch_node_kernel<float>(L, s);
    return cudaGetLastError();
}

template <int T, int B>
static void launch_cell_kernel(const StepLaunch &L, cudaStream_t s) {
    auto *k = L.bido ? (L.ab2 ? cell_kernel<float, T, B, true, true> : cell_kernel<float, T, B, true, false>)
                     : (L.ab2 ? cell_kernel<float, T, B, false, true>
                              : (L.models == (1 << EP_TP06) ? cell_kernel<float, T, B, false, false, 1 << EP_TP06>
                                                            : cell_kernel<float, T, B, false, false>));
    k<<<L.cell_grid, T, 0, s>>>(L.jobs, L.cell_tiles, L.n_cell_tiles, L.done, L.n_jobs);
}

// The staged kernel needs more than the default 48 KB of dynamic shared memory.
static cudaError_t staged_attributes() {
    static std::once_flag once;
    static cudaError_t rc = cudaSuccess;
    std::call_once(once, [] {
        const int full = int(staged::smem_bytes<true>()), part = int(staged::smem_bytes<false>());
        rc = cudaFuncSetAttribute(cell_kernel_staged<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, full);
        if (rc == cudaSuccess)
            rc = cudaFuncSetAttribute(cell_kernel_staged<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, full);
        if (rc == cudaSuccess)
            rc = cudaFuncSetAttribute(cell_kernel_staged<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      part);
        if (rc == cudaSuccess)
            rc = cudaFuncSetAttribute(cell_kernel_staged<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      part);
    });
    return rc;
}

template <bool STATE>
static void launch_staged(const StepLaunch &L, cudaStream_t s) {
    auto *k = L.bido ? cell_kernel_staged<true, STATE> : cell_kernel_staged<false, STATE>;
    k<<<L.cell_grid, kCellThreads, staged::smem_bytes<STATE>(), s>>>(L.jobs, L.cell_tiles, L.n_cell_tiles, L.done,
                                                                     L.n_jobs, L.err);
}

template <class R, int T, int B>
static void launch_fused_kernel(const StepLaunch &L, cudaStream_t s) {
    auto *k = L.bido ? (L.ab2 ? fused_kernel<R, T, B, true, true> : fused_kernel<R, T, B, true, false>)
                     : (L.ab2 ? fused_kernel<R, T, B, false, true> : fused_kernel<R, T, B, false, false>);
    k<<<L.cell_grid, T, 0, s>>>(L.jobs, L.node_tiles, L.cell_tiles, L.work, L.n_work, L.head, L.done, L.n_jobs,
                                L.err);
}

template <class R>
static cudaError_t cell_launch_variant(const StepLaunch &L, cudaStream_t s) {
    if (is_fused_variant(L.cell_variant)) {
        switch (L.cell_variant) {
#define EP_FUSED_CASE(k, T, B)                                                                                 \
    case k:                                                                                                    \
        launch_fused_kernel<R, T, B>(L, s);                                                                    \
        break;
            EP_FUSED_VARIANTS(EP_FUSED_CASE)
#undef EP_FUSED_CASE
        default:
            return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    if (is_staged_variant(L.cell_variant)) {
        if constexpr (std::is_same<R, float>::value) {
            if (!L.ab2 && !L.idx16) {
                cudaError_t e = staged_attributes();
                if (e != cudaSuccess) return e;
                if (L.cell_variant == kStagedVariant) launch_staged<true>(L, s);
                else launch_staged<false>(L, s);
                return cudaGetLastError();
            }
        }
        StepLaunch L0 = L;   // FP64, AB2 or 16-bit indices: the plain variant 0, with its own grid
        L0.cell_variant = 0;
        L0.cell_grid = L.cell_grid0;
        return cell_launch_variant<R>(L0, s);
    }
    // the two-launch shapes: FP64 in kernels_f64.cu; a small FP32 batch with its descriptors as a
    // kernel parameter in kernels_tab.cu (FP32 only: the FP64 step is bound by the FP64 pipe, and its
    // compiled rounding must not depend on the kernel); else the job table in global memory
    if constexpr (std::is_same<R, double>::value) {
        return launch_cell_plain_f64(L, s);
    } else {
        if (tab_eligible(L)) return launch_cell_tab(L, s);
        switch (L.cell_variant) {
#define EP_CELL_CASE(k, T, B)               \
    case k:                                 \
        launch_cell_kernel<T, B>(L, s);     \
        break;
            EP_CELL_VARIANTS(EP_CELL_CASE)
#undef EP_CELL_CASE
        default:
            return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

cudaError_t launch_cell(int precision, const StepLaunch &L, cudaStream_t s) {
    return precision == EP_FP64_PLAIN ? cell_launch_variant<double>(L, s) : cell_launch_variant<float>(L, s);
}

template <class R>
static int cell_blocks_variant(int variant) {
    int nb = 0;
    if (is_fused_variant(variant)) {
        switch (variant) {
#define EP_FUSED_CASE(k, T, B)                                                                              \
    case k:                                                                                                 \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_kernel<R, T, B, false, false>, T, 0);      \
        break;
            EP_FUSED_VARIANTS(EP_FUSED_CASE)
#undef EP_FUSED_CASE
        }
        return nb < 1 ? 1 : nb;
    }
    if (is_staged_variant(variant)) {
        if (std::is_same<R, float>::value && staged_attributes() == cudaSuccess) {
            if (variant == kStagedVariant)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel_staged<false, true>, kCellThreads,
                                                              staged::smem_bytes<true>());
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel_staged<false, false>, kCellThreads,
                                                              staged::smem_bytes<false>());
        }
        if (nb >= 1) return nb;
        variant = 0;
    }
    if constexpr (std::is_same<R, double>::value) {
        return cell_blocks_plain_f64(variant);
    } else {
        switch (variant) {
#define EP_CELL_CASE(k, T, B)                                                                             \
    case k:                                                                                               \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<float, T, B, false, false>, T, 0); \
        break;
            EP_CELL_VARIANTS(EP_CELL_CASE)
#undef EP_CELL_CASE
        }
        return nb < 1 ? 1 : nb;
    }
}

int cell_variant_threads(int variant) {
    switch (variant) {
#define EP_CELL_CASE(k, T, B) \
    case k:                   \
        return T;
        EP_CELL_VARIANTS(EP_CELL_CASE)
        EP_FUSED_VARIANTS(EP_CELL_CASE)
#undef EP_CELL_CASE
    }
    return is_staged_variant(variant) ? kCellThreads : 0;
}

cudaError_t launch_check_finite(int precision, const DevJob *job, long long n_cells, unsigned *count,
                                cudaStream_t s) {
    if (precision == EP_FP64_PLAIN) finite_kernel<double><<<grid_for(n_cells, 256), 256, 0, s>>>(job, n_cells, count);
    else finite_kernel<float><<<grid_for(n_cells, 256), 256, 0, s>>>(job, n_cells, count);
    return cudaGetLastError();
}

int cell_blocks_per_sm(int precision, int variant) {
    return precision == EP_FP64_PLAIN ? cell_blocks_variant<double>(variant) : cell_blocks_variant<float>(variant);
}

int node_blocks_per_sm(int precision) {
    int nb = 0;
    if (precision == EP_FP64_PLAIN)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, node_kernel<double, 2>, kNodeThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, node_kernel<float, 2>, kNodeThreads, 0);
    return nb < 1 ? 1 : nb;
}

// ---------------------------------------------------------------------------
// Step variant that allocates nothing.
//
// Some callers must not allocate device memory while they step a job: a
// process whose device memory is already fully reserved by another runtime's
// memory pool (a new cudaMalloc would fail or fragment that pool), or a
// latency-critical loop that may not call cudaMalloc/cudaFree because those
// can take a global lock or synchronise the device. The variant below keeps
// everything the step needs beyond the job's own arrays -- the job's
// descriptor, its node and cell tile tables, the ticket counter that
// advances the step, and the node values of S1 -- in this file-scope array
// instead of memory allocated per batch, and then runs the very kernels
// ep_step runs, so the results are the same bit for bit. Every GPU that loads
// the library holds the array until the process exits. All calls share it
// and it keeps the last call's contents: calls that overlap on the GPU
// (different streams, threads or contexts on one device) race on it and must
// be serialised by the caller.
//
// Layout: [0, 256) the ticket and the work counter; the descriptor; the node
// tiles; the cell tiles; the work list; the node values (each part 256-byte
// aligned).
namespace noalloc {
constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kMaxNodeTiles = (EP_NOALLOC_MAX_NODES + kNodeThreads - 1) / kNodeThreads;
constexpr size_t kMaxCellTiles = (EP_NOALLOC_MAX_CELLS + kCellThreads - 1) / kCellThreads + EP_N_MODELS;
constexpr size_t kJob = 256;
constexpr size_t kNodeTiles = kJob + round256(sizeof(DevJob));
constexpr size_t kCellTiles = kNodeTiles + round256(kMaxNodeTiles * sizeof(Tile));
constexpr size_t kWork = kCellTiles + round256(kMaxCellTiles * sizeof(Tile));
constexpr size_t kVn = kWork + round256((kMaxNodeTiles + kMaxCellTiles) * sizeof(Work));
constexpr size_t kBytes = kVn + size_t(EP_NOALLOC_MAX_NODES) * sizeof(double);
}  // namespace noalloc
static __device__ __align__(256) unsigned char g_noalloc_scratch[noalloc::kBytes];

// Device address of g_noalloc_scratch, looked up once per CUDA context with
// that context current (in host code the symbol's name is only a host-side
// stand-in). The cache is keyed on the context's unique id, so a context
// re-created after cudaDeviceReset looks the address up again instead of
// reusing one from the context it replaced.
struct NoAllocAddr {
    unsigned long long ctx_id;
    void *p;
};
static NoAllocAddr g_noalloc_addr[64];
static int g_noalloc_n = 0;
static std::mutex g_noalloc_mutex;

// Unique id of the calling thread's current context (cuCtxGetId, reached
// through the runtime's driver entry point so the library needs no link
// against the driver library).
static cudaError_t current_context_id(unsigned long long *id) {
    using CtxGetId = int (*)(void *, unsigned long long *);
    static CtxGetId fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetId>(p);
    });
    if (!fn) return cudaErrorNotSupported;
    if (fn(nullptr, id) == 0) return cudaSuccess;
    // no context current on this thread yet: make the device's primary one current
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    return fn(nullptr, id) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

static cudaError_t noalloc_scratch_address(void **out) {
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    for (int k = 0; k < g_noalloc_n; ++k)
        if (g_noalloc_addr[k].ctx_id == id) {
            *out = g_noalloc_addr[k].p;
            return cudaSuccess;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // contexts are rarely re-created; past 64 the oldest entry is replaced
    const int slot = g_noalloc_n < 64 ? g_noalloc_n++ : int(id % 64);
    g_noalloc_addr[slot] = NoAllocAddr{id, p};
    *out = p;
    return cudaSuccess;
}

cudaError_t launch_step_noalloc(int precision, const DevJob &job, const Tile *node_tiles, int n_node_tiles,
                                const Tile *cell_tiles, int n_cell_tiles, const Work *work, int n_work,
                                int cell_variant, int sm_count, unsigned *err, long long n_steps, cudaStream_t s) {
    using namespace noalloc;
    if (job.n_nodes < 1 || job.n_nodes > EP_NOALLOC_MAX_NODES || job.n_cells < 1 ||
        job.n_cells > EP_NOALLOC_MAX_CELLS || n_node_tiles > int(kMaxNodeTiles) ||
        n_cell_tiles > int(kMaxCellTiles) || n_work > int(kMaxNodeTiles + kMaxCellTiles) ||
        (is_fused_variant(cell_variant) && n_work != n_node_tiles + n_cell_tiles))
        return cudaErrorInvalidValue;
    void *base = nullptr;
    cudaError_t e = noalloc_scratch_address(&base);
    if (e != cudaSuccess) return e;
    unsigned char *b = static_cast<unsigned char *>(base);
    DevJob dj = job;
    dj.vn = b + kVn;
    // the descriptor and the tile tables (host copies, stream-ordered); the ticket must
    // start at zero -- the array keeps whatever the last call left
    e = cudaMemcpyAsync(b + kJob, &dj, sizeof(DevJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + kNodeTiles, node_tiles, size_t(n_node_tiles) * sizeof(Tile), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + kCellTiles, cell_tiles, size_t(n_cell_tiles) * sizeof(Tile), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess && n_work > 0)
        e = cudaMemcpyAsync(b + kWork, work, size_t(n_work) * sizeof(Work), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    StepLaunch L{};
    L.jobs = reinterpret_cast<const DevJob *>(b + kJob);
    L.n_jobs = 1;
    L.node_tiles = reinterpret_cast<const Tile *>(b + kNodeTiles);
    L.n_node_tiles = n_node_tiles;
    L.cell_tiles = reinterpret_cast<const Tile *>(b + kCellTiles);
    L.n_cell_tiles = n_cell_tiles;
    L.done = reinterpret_cast<unsigned *>(b);
    L.head = reinterpret_cast<unsigned *>(b) + 1;
    L.work = reinterpret_cast<const Work *>(b + kWork);
    L.n_work = n_work;
    L.cell_variant = cell_variant;
    L.idx16 = job.idx16;
    L.sm_count = sm_count;
    JobTab<1> tab1{};   // the descriptor as the FP32 kernels' parameter (copied at each launch)
    tab1.n_jobs = 1;
    tab1.cell_begin[1] = n_cell_tiles;
    tab1.node_begin[1] = n_node_tiles;
    tab1.j[0] = dj;
    L.tab1 = &tab1;
    L.node_form = job.col16;
    L.models = 0;
    for (int m = 0; m < EP_N_MODELS; ++m)
        if (job.reg[m].n > 0) L.models |= 1 << m;
    L.err = err;
    L.node_grid = std::max(1, std::min(n_node_tiles, sm_count * node_blocks_per_sm(precision)));
    L.cell_grid = std::max(1, std::min(n_cell_tiles, sm_count * cell_blocks_per_sm(precision, cell_variant)));
    L.cell_grid0 = std::max(1, std::min(n_cell_tiles, sm_count * cell_blocks_per_sm(precision, 0)));
    for (long long it = 0; it < n_steps; ++it) {
        e = launch_step(precision, L, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ep
