// The plain FP64 step's cell kernel in the two-launch shapes (a translation
// unit of its own: the FP64 cell models take the longest to compile).
#include "cellstep.cuh"

namespace ep {

template <int T, int B>
static void launch_f64(const StepLaunch &L, cudaStream_t s) {
    auto *k = L.bido ? (L.ab2 ? cell_kernel<double, T, B, true, true> : cell_kernel<double, T, B, true, false>)
                     : (L.ab2 ? cell_kernel<double, T, B, false, true>
                              : (L.models == (1 << EP_TP06) ? cell_kernel<double, T, B, false, false, 1 << EP_TP06>
                                                            : cell_kernel<double, T, B, false, false>));
    k<<<L.cell_grid, T, 0, s>>>(L.jobs, L.cell_tiles, L.n_cell_tiles, L.done, L.n_jobs);
}

cudaError_t launch_cell_plain_f64(const StepLaunch &L, cudaStream_t s) {
    switch (L.cell_variant) {
#define EP_CELL_CASE(k, T, B)       \
    case k:                         \
        launch_f64<T, B>(L, s);     \
        break;
        EP_CELL_VARIANTS(EP_CELL_CASE)
#undef EP_CELL_CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int cell_blocks_plain_f64(int variant) {
    int nb = 0;
    switch (variant) {
#define EP_CELL_CASE(k, T, B)                                                                              \
    case k:                                                                                                \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<double, T, B, false, false>, T, 0); \
        break;
        EP_CELL_VARIANTS(EP_CELL_CASE)
#undef EP_CELL_CASE
    }
    return nb < 1 ? 1 : nb;
}

}  // namespace ep
