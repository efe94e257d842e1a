// Gather-index decoding and node interpolation (S1, Sec. 3.2), shared by the
// monodomain step kernels and the bidomain solve.
#pragma once

#include "devtypes.h"

namespace ep {

// Inverse-distance node value (S1) over the sliced-ELL entries b, b+32, ...
// < e of one node (32-bit cell indices col). The loads of D entries are
// issued before their products are accumulated, so D gathers are in flight
// at once (D = 6: an interior node of a Kuhn mesh has 24 cells, four groups;
// the fastest of 4, 6, 8 and 12 on the B300); the sum is still taken in
// entry order.
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

// The same over 16-bit entries: the cell of entry k is base + col[k].
template <class R, int D = 6>
__device__ __forceinline__ R node_sum16(const R *__restrict__ w, const unsigned short *__restrict__ col, int base,
                                        const R *__restrict__ V, long long b, long long e) {
    R acc = R(0);
    long long k = b;
    for (; k + 32 * (D - 1) < e; k += 32 * D) {
        int c[D];
        R wk[D], v[D];
#pragma unroll
        for (int i = 0; i < D; ++i) c[i] = base + int(col[k + 32 * i]);
#pragma unroll
        for (int i = 0; i < D; ++i) wk[i] = w[k + 32 * i];
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = V[c[i]];
#pragma unroll
        for (int i = 0; i < D; ++i) acc += wk[i] * v[i];
    }
    for (; k < e; k += 32) acc += w[k] * V[base + int(col[k])];
    return acc;
}

// S1 at one node of a job. F: the form of the job's node -> cell entries --
// 0 32-bit, 1 16-bit, 2 either (read from the job).
template <class R, int D = 6, int F = 2>
__device__ __forceinline__ R node_value(const DevJob &J, const R *__restrict__ V, long long node) {
    const R *__restrict__ w = static_cast<const R *>(J.nw);
    const long long s = node >> 5;
    const long long b = J.slice_ptr[s] + (node & 31), e = J.slice_ptr[s + 1];
    if (F == 1 || (F == 2 && J.col16)) return node_sum16<R, D>(w, J.ncol16, J.cbase[s], V, b, e);
    return node_sum<R, D>(w, J.ncol, V, b, e);
}

// The 16-bit form of cell c's gather indices: u holds the eight node
// offsets from base (its run's nbase), o the four neighbour offsets from c.
__device__ __forceinline__ void decode_idx16(const uint4 u, int base, const uint2 o, long long c, int4 &na, int4 &nb,
                                             int4 &nc) {
    na = make_int4(base + int(u.x & 0xffffu), base + int(u.x >> 16), base + int(u.y & 0xffffu),
                   base + int(u.y >> 16));
    nb = make_int4(base + int(u.z & 0xffffu), base + int(u.z >> 16), base + int(u.w & 0xffffu),
                   base + int(u.w >> 16));
    const int ci = int(c);
    // low halves sign-extended through a 16-bit signed value, high halves by an arithmetic shift
    nc = make_int4(ci + int(short(o.x & 0xffffu)), ci + (int(o.x) >> 16), ci + int(short(o.y & 0xffffu)),
                   ci + (int(o.y) >> 16));
}

// The gather indices of cell c: its vertices (na), the vertex of the
// neighbour opposite each face (nb) and the neighbours (nc).
__device__ __forceinline__ void cell_indices(const DevJob &J, long long c, int4 &na, int4 &nb, int4 &nc) {
    if (J.idx16) {
        decode_idx16(J.cidx16[c], J.nbase[c >> 8], J.nbr16[c], c, na, nb, nc);
    } else {
        na = J.nodes_a[c];
        nb = J.nodes_b[c];
        nc = J.nbr[c];
    }
}

}  // namespace ep
