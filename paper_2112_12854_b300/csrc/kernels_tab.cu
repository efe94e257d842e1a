// Step kernels of an FP32 batch of at most kParamJobs jobs (forward Euler,
// monodomain), the jobs' descriptors a kernel parameter (JobTab): the node
// kernel and the cell kernel in every cell_kernel launch shape.
#include <algorithm>

#include "cellstep.cuh"

namespace ep {

// Job of tile t of a batch whose descriptors are a kernel parameter: t and
// the tile bounds are uniform over the block, so the job index is too, and
// the descriptor's fields are read as uniform constant-bank operands.
template <int K>
__device__ __forceinline__ int tab_job(const JobTab<K> &tab, const int *begin, int t) {
    int j = 0;
#pragma unroll
    for (int k = 1; k < K; ++k) j += (k < tab.n_jobs && t >= begin[k]) ? 1 : 0;
    return j;
}

// node_kernel for an FP32 batch of at most kParamJobs jobs, their
// descriptors a kernel parameter (JobTab).
template <class R, int F, int K>
__global__ void __launch_bounds__(kNodeThreads) node_kernel_tab(const __grid_constant__ JobTab<K> tab,
                                                                const Tile *__restrict__ tiles, int n_tiles) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const DevJob &J = tab.j[tab_job(tab, tab.node_begin, t)];
        const Tile tl = tiles[t];
        const int i = threadIdx.x;
        if (i >= tl.count) continue;
        const long long node = (long long)tl.start + i;
        const long long n = *J.step;
        const R *__restrict__ V = static_cast<const R *>(J.V[n & 1]);
        static_cast<R *>(J.vn)[node] = node_value<R, 6, F>(J, V, node);
    }
}

template <int F>
static void node_tab_impl(const StepLaunch &L, cudaStream_t s) {
    if (L.n_jobs == 1) node_kernel_tab<float, F, 1><<<L.node_grid, kNodeThreads, 0, s>>>(*L.tab1, L.node_tiles,
                                                                                         L.n_node_tiles);
    else node_kernel_tab<float, F, kParamJobs><<<L.node_grid, kNodeThreads, 0, s>>>(*L.tabk, L.node_tiles,
                                                                                   L.n_node_tiles);
}

// Cell kernel for an FP32 batch of at most kParamJobs jobs (forward Euler,
// monodomain), any cell_kernel shape: the jobs' descriptors are a kernel
// parameter (JobTab, __grid_constant__), so the per-cell reads of their
// fields come from the constant bank, as operands that hold no registers,
// instead of the L1 / L2 path of the streamed and gathered data; the TP06
// instance then fits 64 registers without spills. Otherwise cell_kernel: the
// same arithmetic, bitwise the same results.
template <class R, int T, int MINB, int K, int MODELS = 7>
__global__ void __launch_bounds__(T, MINB) cell_kernel_tab(const __grid_constant__ JobTab<K> tab,
                                                            const Tile *__restrict__ tiles, int n_tiles,
                                                            unsigned *done) {
    // one job: its step counter read once (every block reads it before the last one advances it)
    long long n1 = 0;
    if constexpr (K == 1) n1 = *tab.j[0].step;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const DevJob &J = tab.j[tab_job(tab, tab.cell_begin, t)];
        long long n;
        if constexpr (K == 1) n = n1;
        else n = *J.step;
        const R *__restrict__ V = static_cast<const R *>(J.V[n & 1]);
        const Tile tl = tiles[t];
        for (int i = threadIdx.x; i < tl.count; i += T) {
            const long long c = (long long)tl.start + i;
            cell_update_from<R, false, false, false, MODELS>(J, tl.model, c, n, V, global_src<R>(J, tl.model, c, V));
        }
    }
    // Every block has read the step counters; the last one to finish advances them.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            for (int j = 0; j < tab.n_jobs; ++j) *tab.j[j].step += 1;
            *done = 0u;
            __threadfence();
        }
    }
}

// Resident blocks per SM of kernel instance KERN at T threads per block,
// queried once per instance (thread-safe static initialisation).
template <auto KERN, int T>
static int blocks_per_sm_once() {
    static const int nb = [] {
        int q = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, KERN, T, 0);
        return std::max(q, 1);
    }();
    return nb;
}

template <int T, int B, int K>
static void cell_tab_impl(const StepLaunch &L, cudaStream_t s) {
    const bool tt = L.models == (1 << EP_TP06);
    auto *k = tt ? cell_kernel_tab<float, T, B, K, 1 << EP_TP06> : cell_kernel_tab<float, T, B, K>;
    const int nb = tt ? blocks_per_sm_once<cell_kernel_tab<float, T, B, K, 1 << EP_TP06>, T>()
                      : blocks_per_sm_once<cell_kernel_tab<float, T, B, K>, T>();
    const int grid = L.sm_count > 0 ? std::max(1, std::min(L.n_cell_tiles, L.sm_count * nb)) : L.cell_grid;
    if constexpr (K == 1) k<<<grid, T, 0, s>>>(*L.tab1, L.cell_tiles, L.n_cell_tiles, L.done);
    else k<<<grid, T, 0, s>>>(*L.tabk, L.cell_tiles, L.n_cell_tiles, L.done);
}

bool tab_eligible(const StepLaunch &L) {
    return (L.n_jobs == 1 ? L.tab1 != nullptr : L.tabk != nullptr) && !L.bido && !L.ab2;
}

cudaError_t launch_node_tab(const StepLaunch &L, cudaStream_t s) {
    if (L.node_form == 0) node_tab_impl<0>(L, s);
    else if (L.node_form == 1) node_tab_impl<1>(L, s);
    else node_tab_impl<2>(L, s);
    return cudaGetLastError();
}

cudaError_t launch_cell_tab(const StepLaunch &L, cudaStream_t s) {
    switch (L.cell_variant) {
#define EP_CELL_CASE(k, T, B)                                 \
    case k:                                                   \
        if (L.n_jobs == 1) cell_tab_impl<T, B, 1>(L, s);      \
        else cell_tab_impl<T, B, kParamJobs>(L, s);           \
        break;
        EP_CELL_VARIANTS(EP_CELL_CASE)
#undef EP_CELL_CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ep
