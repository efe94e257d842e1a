// Bidomain solve kernel (see bidomain.h): one cooperative, persistent launch
// per job and step runs the whole restarted GMRES solve of the elliptic
// equation -- node values, fluxes, Gram-Schmidt passes, reductions and the
// Givens least-squares update -- with grid barriers between the phases, so
// no host round trip decides the iteration count.
//
// GMRES (Sec. 3.2; textbook restarted GMRES): Arnoldi with classical
// Gram-Schmidt, once (CGS) or twice (CGS2) -- one or two streaming passes
// over the basis and one reduction each, instead of the j dependent
// reductions of modified Gram-Schmidt -- Givens rotations on the Hessenberg
// column, and a restart after `restart` steps from the true residual, which
// also decides convergence. The basis is stored unnormalised with a scale
// per vector, so normalisation needs no extra pass, and is streamed in
// 16-byte vectors. Dot products are summed per thread in the compute type,
// per block and across blocks in FP64, in a fixed order: the result depends
// only on the job and the device, not on the batch.
#include <algorithm>
#include <cmath>

#include "bidomain.h"
#include "nodesum.cuh"

namespace ep {

namespace {

template <class R> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4_32a; };

// 16-byte vectors for the streaming passes over the Krylov basis.
template <class R> struct VW;
template <> struct VW<float> { using type = float4; static constexpr int n = 4; };
template <> struct VW<double> { using type = double2; static constexpr int n = 2; };

constexpr int kWarps = kBidoThreads / 32;
constexpr int KP = kBidoMaxRestart + 1;
constexpr int kShortNP = 13;   // accumulators of the kernel instance for restarts up to 12

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of a cooperative launch (all blocks co-resident). The wait is
// bounded: past limit_ns the block sets the error flag and every block
// leaves the kernel at its next barrier. Returns false on error.
__device__ bool grid_sync(BidoSync *s, int *flag_sh, unsigned long long limit_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &s->gen;
        volatile int *verr = &s->err;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&s->count, 1u) == gridDim.x - 1) {
            atomicExch(&s->count, 0u);
            __threadfence();
            atomicAdd(&s->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g && *verr == 0) {
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(&s->err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *flag_sh = *verr;
    }
    __syncthreads();
    return *flag_sh == 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block partial sums of acc[0..count) into part[i * gridDim.x + blockIdx.x].
template <class R, int N>
__device__ void block_partials(const R (&acc)[N], int count, double *part, double *red_sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < count) {
            const double v = warp_sum(double(acc[i]));
            if (lane == 0) red_sh[warp * KP + i] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red_sh[w * KP + i];
        part[size_t(i) * gridDim.x + blockIdx.x] = s;
    }
}

// Grid totals of the partials (after a barrier), computed by every block in
// the same order: tot_sh[i] for i < count.
__device__ void grid_totals(const double *part, int count, double *tot_sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < count; i += kWarps) {
        double s = 0.0;
        for (int b = lane; b < int(gridDim.x); b += 32) s += part[size_t(i) * gridDim.x + b];
        s = warp_sum(s);
        if (lane == 0) tot_sh[i] = s;
    }
    __syncthreads();
}

// S1 on a field x (times `scale`): inverse-distance node values into vn.
template <class R>
__device__ void node_pass(const DevJob &J, const R *__restrict__ x, R scale, R *__restrict__ vn, long long gtid,
                          long long gsz) {
    for (long long node = gtid; node < J.n_nodes; node += gsz) {
        // one entry per iteration: in this kernel (80 registers, three blocks per SM) six-deep
        // gathers made the node phase slower (3.13 against 2.65 ms per step on the 9.6M-cell wedge)
        vn[node] = node_value<R, 1>(J, x, node) * scale;
    }
}

// Folded diffusion term (Eqs. 7-8) of cell c for the field x * scale whose
// node values are vn, with coefficient set (wa, wb, q).
template <class R>
__device__ __forceinline__ R flux(const DevJob &J, const void *wa_, const void *wb_, const void *q_,
                                  const R *__restrict__ vn, const R *__restrict__ x, R scale, long long c) {
    using R4 = typename V4<R>::type;
    int4 na, nb, nc;
    cell_indices(J, c, na, nb, nc);
    const R4 wa = static_cast<const R4 *>(wa_)[c];
    const R4 wb = static_cast<const R4 *>(wb_)[c];
    const R4 q = static_cast<const R4 *>(q_)[c];
    const R xc = x[c];
    R d = wa.x * vn[na.x] + wa.y * vn[na.y] + wa.z * vn[na.z] + wa.w * vn[na.w];
    d += wb.x * vn[nb.x] + wb.y * vn[nb.y] + wb.z * vn[nb.z] + wb.w * vn[nb.w];
    d += scale * (q.x * (x[nc.x] - xc) + q.y * (x[nc.y] - xc) + q.z * (x[nc.z] - xc) + q.w * (x[nc.w] - xc));
    return d;
}

}  // namespace

// Resident blocks per SM the register budget is cut for: three for FP32
// (80 registers, 24 warps per SM to keep the gathers of the flux passes in
// flight), one for FP64.
template <class R> struct BidoMinBlocks { static constexpr int value = 1; };
template <> struct BidoMinBlocks<float> { static constexpr int value = 3; };

// NP: the per-thread dot-product accumulators and basis vectors the passes
// are unrolled for (restart + 1 at most): 13 for the default restart of 12,
// which keeps the accumulators of longer restarts out of the registers, or
// kBidoMaxRestart + 1.
template <class R, int NP>
__global__ void __launch_bounds__(kBidoThreads, BidoMinBlocks<R>::value)
    bido_kernel(const __grid_constant__ BidoArgs A) {
    __shared__ double red_sh[kWarps * KP];
    __shared__ double tot[KP];
    __shared__ double H[KP * kBidoMaxRestart];   // H[i * kBidoMaxRestart + j]
    __shared__ double cs[kBidoMaxRestart], sn[kBidoMaxRestart], g[KP], y[KP];
    __shared__ double sc[KP];                     // basis vector i = basis_i * sc[i]
    __shared__ R coef[KP];                        // per-pass multipliers of the basis vectors
    __shared__ int flag_sh;

    const DevJob &J = A.job;   // constant bank: the per-cell reads of its fields hold no registers
    const long long n = J.n_cells;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gsz = (long long)gridDim.x * blockDim.x;
    const long long step = *J.step;
    const R *__restrict__ V = static_cast<const R *>(J.V[step & 1]);
    R *__restrict__ vn = static_cast<R *>(J.vn);
    R *__restrict__ x = static_cast<R *>(A.ve);
    R *__restrict__ b = static_cast<R *>(A.b);
    R *__restrict__ wv = static_cast<R *>(A.w);
    R *__restrict__ basis = static_cast<R *>(A.basis);
    const long long ld = A.ld;
    // vector views (ld is a multiple of 64; the pads past n_cells stay zero)
    using VT = typename VW<R>::type;
    constexpr int NW = VW<R>::n;
    const long long lq = ld / NW;
    const VT *__restrict__ bq = reinterpret_cast<const VT *>(basis);
    VT *__restrict__ wq = reinterpret_cast<VT *>(wv);
    const int m = A.restart;
    R acc[NP];
    // Two partial-sum buffers used in turn: a block may write the next
    // reduction's partials while another still reads the previous totals, but
    // never before every block has passed the barrier that follows.
    int red = 0;
    auto part_w = [&]() { return A.part + size_t(red & 1) * KP * gridDim.x; };
    // device time between barriers, by phase (block 0's clock): 0 node values,
    // 1 fluxes (+ first dots), 2 second Gram-Schmidt pass, 3 third pass,
    // 4 updates of x and the gauge
    __shared__ unsigned long long ph_sh[5], t_last_sh;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) ph_sh[k] = 0ull;
        t_last_sh = global_ns();
    }
#define BIDO_SYNC(ph)                                          \
    do {                                                       \
        if (!grid_sync(A.sync, &flag_sh, A.barrier_limit_ns)) { \
            if (threadIdx.x == 0) {                            \
                A.stats->timeout = 1;                          \
                A.stats->hist = 0;                             \
            }                                                  \
            return;                                            \
        }                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0) {             \
            const unsigned long long t_ = global_ns();         \
            ph_sh[ph] += t_ - t_last_sh;                       \
            t_last_sh = t_;                                    \
        }                                                      \
    } while (0)

    long long iters = 0;
    int failed = 0;
    double res = 0.0, bnorm = 0.0;
    // algorithmic bytes of each phase: every array it touches counted once
    // (the node table as stored, coefficients, indices, fields, basis vectors)
    const double RB = double(sizeof(R)), dn = double(n), dnn = double(J.n_nodes);
    const double IB = J.idx16 ? 2.0 : 4.0;   // bytes of one stored gather index
    const double node_b = double(J.slice_ptr[(J.n_nodes + 31) >> 5]) * (IB + RB) + dn * RB + dnn * RB;
    const double flux_b = dn * (12.0 * IB + 12.0 * RB) + dnn * RB + 2.0 * dn * RB;
    double bytes = 0.0;
    if (A.mode == 0) {
        // right-hand side b = -L_i(V^{n+1}) and its norm
        node_pass<R>(J, V, R(1), vn, gtid, gsz);
        BIDO_SYNC(0);
        // initial guess: v_e^n, or 2 v_e^n - v_e^{n-1} once two consecutive solutions are held
        // (a first-order extrapolation in time; the gauge of both is the same)
        const int hist = A.stats->hist;
        R *__restrict__ vp = static_cast<R *>(A.vprev);
        acc[0] = R(0);
        for (long long c = gtid; c < n; c += gsz) {
            const R bc = -flux<R>(J, J.wa, J.wb, J.q, vn, V, R(1), c);
            b[c] = bc;
            acc[0] += bc * bc;
            if (hist >= 2) {
                const R xc = x[c];
                x[c] = R(2) * xc - vp[c];
                vp[c] = xc;
            } else if (hist == 1) {
                vp[c] = x[c];
            }
        }
        block_partials<R, NP>(acc, 1, part_w(), red_sh);
        BIDO_SYNC(1);
        grid_totals(part_w(), 1, tot);
        ++red;
        bnorm = sqrt(tot[0]);
        bytes += node_b + flux_b;
        const double thr = fmax(A.tol * bnorm, A.atol * sqrt(double(n)));
        for (;;) {
            // true residual r = b - L_ie x into basis vector 0
            node_pass<R>(J, x, R(1), vn, gtid, gsz);
            BIDO_SYNC(0);
            acc[0] = R(0);
            for (long long c = gtid; c < n; c += gsz) {
                const R r = b[c] - flux<R>(J, A.wa, A.wb, A.q, vn, x, R(1), c);
                basis[c] = r;
                acc[0] += r * r;
            }
            block_partials<R, NP>(acc, 1, part_w(), red_sh);
            BIDO_SYNC(1);
            grid_totals(part_w(), 1, tot);
            ++red;
            const double beta = sqrt(tot[0]);
            res = beta;
            bytes += node_b + flux_b + dn * RB;
            if (beta <= thr) break;
            if (iters >= A.max_iter) {
                failed = 1;
                break;
            }
            if (threadIdx.x == 0) {
                sc[0] = 1.0 / beta;
                for (int i = 0; i < NP; ++i) g[i] = 0.0;
                g[0] = beta;
            }
            __syncthreads();
            int j = 0;
            while (j < m && iters < A.max_iter) {
                const R *__restrict__ vj = basis + j * ld;
                const R sj = R(sc[j]);
                // w = L_ie v_j, and the first Gram-Schmidt dots <v_i, w>
                node_pass<R>(J, vj, sj, vn, gtid, gsz);
                BIDO_SYNC(0);
#pragma unroll
                for (int i = 0; i < NP; ++i) acc[i] = R(0);
                for (long long c = gtid; c < n; c += gsz) {
                    const R w = flux<R>(J, A.wa, A.wb, A.q, vn, vj, sj, c);
                    wv[c] = w;
#pragma unroll
                    for (int i = 0; i < NP; ++i)
                        if (i <= j) acc[i] += basis[i * ld + c] * w;
                }
                block_partials<R, NP>(acc, j + 1, part_w(), red_sh);
                BIDO_SYNC(1);
                grid_totals(part_w(), j + 1, tot);
                ++red;
                if (threadIdx.x <= j) {
                    const double h = tot[threadIdx.x] * sc[threadIdx.x];
                    H[threadIdx.x * kBidoMaxRestart + j] = h;
                    coef[threadIdx.x] = R(h * sc[threadIdx.x]);
                }
                __syncthreads();
                if (A.reorth) {
                    // second pass: w' = w - V h, and the re-orthogonalisation dots
#pragma unroll
                    for (int i = 0; i < NP; ++i) acc[i] = R(0);
                    for (long long qi = gtid; qi < lq; qi += gsz) {
                        VT w = wq[qi];
                        R *wp = reinterpret_cast<R *>(&w);
#pragma unroll
                        for (int i = 0; i < NP; ++i)
                            if (i <= j) {
                                const VT b4 = bq[i * lq + qi];
                                const R *bp = reinterpret_cast<const R *>(&b4);
                                const R ci = coef[i];
#pragma unroll
                                for (int k = 0; k < NW; ++k) wp[k] -= ci * bp[k];
                            }
                        wq[qi] = w;
#pragma unroll
                        for (int i = 0; i < NP; ++i)
                            if (i <= j) {
                                const VT b4 = bq[i * lq + qi];
                                const R *bp = reinterpret_cast<const R *>(&b4);
                                R d = R(0);
#pragma unroll
                                for (int k = 0; k < NW; ++k) d += bp[k] * wp[k];
                                acc[i] += d;
                            }
                    }
                    block_partials<R, NP>(acc, j + 1, part_w(), red_sh);
                    BIDO_SYNC(2);
                    grid_totals(part_w(), j + 1, tot);
                    ++red;
                    if (threadIdx.x <= j) {
                        const double h2 = tot[threadIdx.x] * sc[threadIdx.x];
                        H[threadIdx.x * kBidoMaxRestart + j] += h2;
                        coef[threadIdx.x] = R(h2 * sc[threadIdx.x]);
                    }
                    __syncthreads();
                }
                // last pass: v_{j+1} (unnormalised) = w - V (coefficients of the last
                // projection), and its norm
                VT *__restrict__ vq = reinterpret_cast<VT *>(basis + (j + 1) * ld);
                acc[0] = R(0);
                for (long long qi = gtid; qi < lq; qi += gsz) {
                    VT w = wq[qi];
                    R *wp = reinterpret_cast<R *>(&w);
#pragma unroll
                    for (int i = 0; i < NP; ++i)
                        if (i <= j) {
                            const VT b4 = bq[i * lq + qi];
                            const R *bp = reinterpret_cast<const R *>(&b4);
                            const R ci = coef[i];
#pragma unroll
                            for (int k = 0; k < NW; ++k) wp[k] -= ci * bp[k];
                        }
                    vq[qi] = w;
#pragma unroll
                    for (int k = 0; k < NW; ++k) acc[0] += wp[k] * wp[k];
                }
                block_partials<R, NP>(acc, 1, part_w(), red_sh);
                BIDO_SYNC(3);
                grid_totals(part_w(), 1, tot);
                ++red;
                const double hn = sqrt(tot[0]);
                bytes += node_b + flux_b + (A.reorth ? double(3 * (j + 1) + 4) : double(2 * (j + 1) + 2)) * dn * RB;
                if (threadIdx.x == 0) {
                    sc[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
                    double *Hc = H + j;   // column j, row stride kBidoMaxRestart
                    for (int i = 0; i < j; ++i) {
                        const double a = Hc[i * kBidoMaxRestart], c2 = Hc[(i + 1) * kBidoMaxRestart];
                        Hc[i * kBidoMaxRestart] = cs[i] * a + sn[i] * c2;
                        Hc[(i + 1) * kBidoMaxRestart] = -sn[i] * a + cs[i] * c2;
                    }
                    const double a = Hc[j * kBidoMaxRestart];
                    const double rr = sqrt(a * a + hn * hn);
                    cs[j] = rr > 0.0 ? a / rr : 1.0;
                    sn[j] = rr > 0.0 ? hn / rr : 0.0;
                    Hc[j * kBidoMaxRestart] = rr;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                }
                __syncthreads();
                ++j;
                ++iters;
                if (fabs(g[j]) <= thr || hn == 0.0) break;
            }
            // x += V_j y with H_j y = g (upper triangular, every block the same)
            if (threadIdx.x == 0) {
                for (int i = j - 1; i >= 0; --i) {
                    double s = g[i];
                    for (int l = i + 1; l < j; ++l) s -= H[i * kBidoMaxRestart + l] * y[l];
                    const double d = H[i * kBidoMaxRestart + i];
                    y[i] = d != 0.0 ? s / d : 0.0;
                }
                for (int i = 0; i < j; ++i) coef[i] = R(y[i] * sc[i]);
            }
            __syncthreads();
            bytes += double(2 + j) * dn * RB;
            VT *__restrict__ xq = reinterpret_cast<VT *>(x);
            for (long long qi = gtid; qi < lq; qi += gsz) {
                VT xv = xq[qi];
                R *xp = reinterpret_cast<R *>(&xv);
#pragma unroll
                for (int i = 0; i < NP; ++i)
                    if (i < j) {
                        const VT b4 = bq[i * lq + qi];
                        const R *bp = reinterpret_cast<const R *>(&b4);
                        const R ci = coef[i];
#pragma unroll
                        for (int k = 0; k < NW; ++k) xp[k] += ci * bp[k];
                    }
                xq[qi] = xv;
            }
            BIDO_SYNC(4);
        }
        // gauge: zero volume-weighted mean
        const R *__restrict__ wvol = static_cast<const R *>(A.wvol);
        acc[0] = R(0);
        for (long long c = gtid; c < n; c += gsz) acc[0] += wvol[c] * x[c];
        block_partials<R, NP>(acc, 1, part_w(), red_sh);
        BIDO_SYNC(4);
        grid_totals(part_w(), 1, tot);
        ++red;
        const R mean = R(tot[0]);
        bytes += 4.0 * dn * RB;
        for (long long c = gtid; c < n; c += gsz) x[c] -= mean;
        BIDO_SYNC(4);
    }
    // intracellular flux of v_e for the next step's V update
    node_pass<R>(J, x, R(1), vn, gtid, gsz);
    BIDO_SYNC(0);
    R *__restrict__ xd = static_cast<R *>(A.xdiv);
    for (long long c = gtid; c < n; c += gsz) xd[c] = flux<R>(J, J.wa, J.wb, J.q, vn, x, R(1), c);
    if (A.mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) A.stats->hist = 1;   // v_e set from outside
    if (A.mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        BidoStats *st = A.stats;
        st->hist = st->hist < 2 ? st->hist + 1 : 2;
        st->last_iters = iters;
        st->total_iters += iters;
        st->solves += 1;
        st->last_res = res;
        st->last_bnorm = bnorm;
        st->failed |= failed;
        st->alg_bytes += bytes + node_b + flux_b;
        ph_sh[1] += global_ns() - t_last_sh;
        for (int k = 0; k < 5; ++k) st->phase_ms[k] += 1e-6 * double(ph_sh[k]);
    }
#undef BIDO_SYNC
}

namespace {

template <class R>
__global__ void field_gather_kernel(const R *__restrict__ src, const int *__restrict__ perm, long long n,
                                    double *__restrict__ out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[perm[c]] = double(src[c]);
}

template <class R>
__global__ void field_scatter_kernel(const double *__restrict__ in, const int *__restrict__ perm, long long n,
                                     R *__restrict__ dst) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) dst[c] = R(in[perm[c]]);
}

// Both accumulator counts of a precision run at the same register budget
// (BidoMinBlocks), so one grid serves both.
template <class R>
int grid_of(int sm_count) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bido_kernel<R, KP>, kBidoThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return sm_count * std::max(1, std::min(nb, 4));
}

}  // namespace

int bido_grid(int precision, int sm_count, long long n_cells) {
    const int co = precision == EP_FP64_PLAIN ? grid_of<double>(sm_count) : grid_of<float>(sm_count);
    const long long want = (n_cells + 4 * kBidoThreads - 1) / (4 * kBidoThreads);
    return int(std::max(1LL, std::min<long long>(co, want)));
}

cudaError_t launch_bido(int precision, const BidoArgs &a, const DevJob &dj, int grid, cudaStream_t s) {
    BidoArgs arg = a;
    arg.job = dj;
    void *args[] = {&arg};
    const cudaError_t e = cudaMemsetAsync(a.sync, 0, sizeof(BidoSync), s);
    if (e != cudaSuccess) return e;
    const bool short_restart = a.restart + 1 <= kShortNP;
    const void *k = precision == EP_FP64_PLAIN
                        ? (short_restart ? reinterpret_cast<const void *>(bido_kernel<double, kShortNP>)
                                         : reinterpret_cast<const void *>(bido_kernel<double, KP>))
                        : (short_restart ? reinterpret_cast<const void *>(bido_kernel<float, kShortNP>)
                                         : reinterpret_cast<const void *>(bido_kernel<float, KP>));
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kBidoThreads), args, 0, s);
}

cudaError_t launch_field_gather(int precision, const void *src, const int *perm, long long n, double *out,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = unsigned((n + 255) / 256);
    if (precision == EP_FP64_PLAIN)
        field_gather_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(src), perm, n, out);
    else
        field_gather_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(src), perm, n, out);
    return cudaGetLastError();
}

cudaError_t launch_field_scatter(int precision, const double *in, const int *perm, long long n, void *dst,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = unsigned((n + 255) / 256);
    if (precision == EP_FP64_PLAIN)
        field_scatter_kernel<double><<<blocks, 256, 0, s>>>(in, perm, n, static_cast<double *>(dst));
    else
        field_scatter_kernel<float><<<blocks, 256, 0, s>>>(in, perm, n, static_cast<float *>(dst));
    return cudaGetLastError();
}

}  // namespace ep
