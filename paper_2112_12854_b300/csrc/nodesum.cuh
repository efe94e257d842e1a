// Node interpolation (S1, Sec. 3.2) over the sliced-ELL node -> cell table,
// shared by the monodomain node kernels and the bidomain solve's node passes.
#pragma once

namespace ep {

// Inverse-distance node value (S1) over the sliced-ELL entries b, b+32, ...
// < e of one node. The loads of D entries are issued before their products
// are accumulated, so D gathers are in flight at once (D = 6: an interior
// node of a Kuhn mesh has 24 cells, four groups; the fastest of 4, 6, 8 and
// 12 on the B300); the sum is still taken in entry order.
template <class R, int D = 6>
__device__ __forceinline__ R node_sum(const R *__restrict__ w, const int *__restrict__ col, const R *__restrict__ V,
                                      long long b, long long e) {
    R acc = R(0);
    long long k = b;
    for (; k + 32 * (D - 1) < e; k += 32 * D) {
        int c[D];
        R wk[D], v[D];
#pragma unroll
        for (int i = 0; i < D; ++i) c[i] = col[k + 32 * i];
#pragma unroll
        for (int i = 0; i < D; ++i) wk[i] = w[k + 32 * i];
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = V[c[i]];
#pragma unroll
        for (int i = 0; i < D; ++i) acc += wk[i] * v[i];
    }
    for (; k < e; k += 32) acc += w[k] * V[col[k]];
    return acc;
}

}  // namespace ep
