// Device code of one cell's step (Sec. 3.2), shared by the step kernels of
// kernels.cu, kernels_tab.cu and kernels_f64.cu: the stimulus of Eq. 4, the
// junction terms of Sec. 3.3, the diffusion term of Eqs. 7-8 from the
// folded coefficients, the cell model, V^{n+1} and the activation time; and
// cell_kernel, the persistent cell kernel over a batch's job table.
#pragma once
#include <cmath>

#include "crncell.cuh"
#include "kernels.h"
#include "nodesum.cuh"
#include "ttcells.cuh"
#include "varmap.h"

namespace ep {

// In-place state access of local cell i of a region.
template <class R>
__device__ __forceinline__ CellIO<R> region_io(const DevRegion &rg, long long i) {
    R *x = static_cast<R *>(rg.r) + i;
    double *a = rg.a + i;
    return CellIO<R>{x, a, rg.stride, x, a, rg.stride};
}

template <class R> struct Vec4T;
template <> struct Vec4T<float> { using type = float4; };
template <> struct Vec4T<double> { using type = double4_32a; };

template <class R>
__device__ __forceinline__ R stimulus(const DevJob &J, unsigned mask, long long n) {
    R is = R(0);
    for (int k = 0; k < J.n_stim; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const DevStim &s = J.stim[k];
        bool on;
        if (n < s.n_on) on = false;
        else if (s.n_per <= 0) on = n < s.n_on + s.n_dur;
        else on = ((n - s.n_on) % s.n_per) < s.n_dur;
        if (on) is += pick<R>(s.amp, s.amp_f);
    }
    return is;
}

__device__ __forceinline__ bool window_on(double t_trig, double delay, double dur, double t) {
    return t_trig > -INFINITY && t >= t_trig + delay && t < t_trig + delay + dur;
}

// Junction terms of a cell touched by the conduction graph (Sec. 3.3): the
// resistive current g_cell (V_m - V_p) and the triggered stimulus. The
// cell's (cell, junction) entries are found by binary search.
template <class R>
__device__ void junction_cell_terms(const DevJob &J, long long c, long long n, R Vc, R &is, R &ix, int &first,
                                    int &last) {
    const DevGraph &G = J.g;
    int lo = 0, hi = G.n_tgt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (G.tgt_cell[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    first = lo;
    const R *Vg = static_cast<const R *>(G.V[n & 1]);
    const double t = double(n) * J.dt;
    int k = lo;
    for (; k < G.n_tgt && G.tgt_cell[k] == c; ++k) {
        const int e = G.tgt_junc[k], j = e & (kJunctionSource - 1);
        if (e & kJunctionSource) {   // source of a cell-to-cell node, excited back (two-way)
            if (G.two_way && window_on(G.t_cell[j], G.delay_anti, G.duration, t))
                is += pick<R>(G.amplitude, G.amplitude_f);
        } else if (G.jmode[j] == EP_PMJ_RESISTIVE) {
            ix += pick<R>(G.g_cell, G.g_cell_f) * (Vc - Vg[G.jnode[j]]);
        } else if (window_on(G.t_graph[j], G.delay_ortho, G.duration, t)) {
            is += pick<R>(G.amplitude, G.amplitude_f);
        }
    }
    last = k;
}

// Muscle-side threshold crossing of two-way triggered junctions.
template <class R>
__device__ void junction_cell_crossing(const DevJob &J, long long c, long long n, R v0, R v1, int first, int last) {
    const DevGraph &G = J.g;
    const double th = G.threshold;
    if (!(double(v0) < th && double(v1) >= th)) return;
    const double tc = double(n) * J.dt + J.dt * (th - double(v0)) / (double(v1) - double(v0));
    for (int k = first; k < last; ++k) {
        const int e = G.tgt_junc[k], j = e & (kJunctionSource - 1);
        if (e & kJunctionSource) G.t_graph[j] = tc;   // the source cell of a cell-to-cell node fires
        else if (G.two_way && G.jmode[j] != EP_PMJ_RESISTIVE && G.jcell[j] == c) G.t_cell[j] = tc;
    }
}

// A cell's streamed step inputs: its gather indices (decoded), and where the
// rest is read -- straight from the job's arrays in global memory, or from a
// shared-memory stage filled by bulk copies (cell_kernel_staged). The
// gathered inputs (node values, neighbour potentials) are always read from
// global memory.
template <class R>
struct CellSrc {
    int4 na, nb, nc;
    const typename Vec4T<R>::type *wa, *wb, *q;
    const R *Vc;
    const uint8_t *smask, *pset;
    CellIO<R> io;
};

template <class R>
__device__ __forceinline__ CellSrc<R> global_src(const DevJob &J, int model, long long c, const R *V) {
    using R4 = typename Vec4T<R>::type;
    const DevRegion &rg = J.reg[model];
    int4 na, nb, nc;
    cell_indices(J, c, na, nb, nc);
    return CellSrc<R>{na, nb, nc, static_cast<const R4 *>(J.wa) + c, static_cast<const R4 *>(J.wb) + c,
                      static_cast<const R4 *>(J.q) + c, V + c, J.smask + c, J.pset + c,
                      region_io<R>(rg, c - rg.off)};
}

// Node value k for the cell update. In the fused kernel, where other warps
// of the same launch write the node values, the loads are plain weak loads
// (ld.global.ca), never the non-coherent read-only path: they follow the
// warp's acquire of the node tiles, and a line of node values is first
// loaded in a launch only after its tile is complete.
template <class R, bool CG>
__device__ __forceinline__ R node_at(const R *vn, int k) {
    if constexpr (CG) return __ldca(vn + k);
    else return vn[k];
}

// XD: the batch holds bidomain jobs, whose cells add L_i(v_e^n) (first line
// of Eq. 6) to the diffusion term; AB2: the batch holds jobs that advance the
// non-gating variables by second-order Adams-Bashforth. Batches without them
// compile without the code. CG: the node values come from the same launch.
// MODELS: the cell models a batch holds (bit m for model m); a batch of TP06
// cells only compiles TP06 alone, whose register demand is lower.
template <class R, bool XD = false, bool AB2 = false, bool CG = false, int MODELS = 7>
__device__ __forceinline__ void cell_update_from(const DevJob &J, int model, long long c, long long n, const R *V,
                                                 const CellSrc<R> &src) {
    using R4 = typename Vec4T<R>::type;
    R *__restrict__ Vnext = static_cast<R *>(J.V[(n & 1) ^ 1]);
    const R *vn = static_cast<const R *>(J.vn);
    const int4 na = src.na, nb = src.nb, nc = src.nc;
    const R4 wa = *src.wa;
    const R4 wb = *src.wb;
    const R4 q = *src.q;
    const R Vc = *src.Vc;
    // diffusion term of Eq. 7 (S2 + S3 folded): eight node values, four neighbours
    R diff = wa.x * node_at<R, CG>(vn, na.x) + wa.y * node_at<R, CG>(vn, na.y) + wa.z * node_at<R, CG>(vn, na.z) +
             wa.w * node_at<R, CG>(vn, na.w);
    diff += wb.x * node_at<R, CG>(vn, nb.x) + wb.y * node_at<R, CG>(vn, nb.y) + wb.z * node_at<R, CG>(vn, nb.z) +
            wb.w * node_at<R, CG>(vn, nb.w);
    diff += q.x * (V[nc.x] - Vc) + q.y * (V[nc.y] - Vc) + q.z * (V[nc.z] - Vc) + q.w * (V[nc.w] - Vc);
    if (XD && J.xdiv) diff += static_cast<const R *>(J.xdiv)[c];

    const unsigned mask = *src.smask;
    R is = mask ? stimulus<R>(J, mask, n) : R(0);
    const unsigned ps = *src.pset;
    R ix = R(0);
    int jfirst = 0, jlast = 0;
    if (ps & kJunctionFlag) junction_cell_terms<R>(J, c, n, Vc, is, ix, jfirst, jlast);
    const DevParams &P = J.params[ps & (EP_MAX_PARAM_SETS - 1)];
    const R dt = pick<R>(J.dt, J.dt_f);
    R iion;
    Rates<R, AB2> rt;
    if constexpr (AB2) {
        if (J.integrator == EP_INTEGRATOR_AB2) {
            const DevRegion &rg = J.reg[model];
            rt.h = static_cast<R *>(rg.h) + (c - rg.off);
            rt.st = rg.stride;
            rt.on = n > J.ab2_from;
        }
    }
    if constexpr (MODELS == (1 << EP_TP06)) {
        iion = tt_step<R, false, AB2>(src.io, P, Vc, dt, is, rt);
    } else {
        if (model == EP_TP06) iion = tt_step<R, false, AB2>(src.io, P, Vc, dt, is, rt);
        else if (model == EP_STEWART) iion = tt_step<R, true, AB2>(src.io, P, Vc, dt, is, rt);
        else iion = crn_step<R, AB2>(src.io, P, Vc, dt, rt);
    }
    const R Vn = Vc + dt * rt(0, diff - iion - is - ix);
    Vnext[c] = Vn;
    if ((ps & kJunctionFlag) && (J.g.two_way || J.g.cell_nodes)) junction_cell_crossing<R>(J, c, n, Vc, Vn, jfirst, jlast);
    const R th = pick<R>(J.threshold, J.threshold_f);
    if (Vc < th && Vn >= th) {
        R *act = static_cast<R *>(J.act);
        if (isinf(act[c])) act[c] = R(double(n) * J.dt) + dt * (th - Vc) / (Vn - Vc);
    }
}

template <class R, bool XD = false, bool AB2 = false, bool CG = false, int MODELS = 7>
__device__ __forceinline__ void cell_update(const DevJob &J, int model, long long c) {
    const long long n = *J.step;
    const R *__restrict__ V = static_cast<const R *>(J.V[n & 1]);
    cell_update_from<R, XD, AB2, CG, MODELS>(J, model, c, n, V, global_src<R>(J, model, c, V));
}

// Launch-shape variants of the cell kernel, chosen by ep_autotune: threads
// per block and the minimum number of resident blocks per SM requested from
// the register allocator. All variants run the same per-cell arithmetic, so
// their results are bitwise identical. Tiles hold kCellThreads cells; a
// block narrower than a tile walks it in strides of its width.
template <class R, int T, int MINB, bool XD, bool AB2, int MODELS = 7>
__global__ void __launch_bounds__(T, MINB) cell_kernel(const DevJob *__restrict__ jobs,
                                                        const Tile *__restrict__ tiles, int n_tiles,
                                                        unsigned *done, int n_jobs) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        for (int i = threadIdx.x; i < tl.count; i += T)
            cell_update<R, XD, AB2, false, MODELS>(jobs[tl.job], tl.model, (long long)tl.start + i);
    }
    // Every block has read the step counters; the last one to finish advances them.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            for (int j = 0; j < n_jobs; ++j) *jobs[j].step += 1;
            *done = 0u;
            __threadfence();
        }
    }
}

}  // namespace ep
