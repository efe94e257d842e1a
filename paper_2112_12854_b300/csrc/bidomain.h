// Bidomain extension of a job (Eq. 1, Eqs. 5-6): the extracellular
// potential v_e from the elliptic equation
//     L_ie(v_e^{n+1}) = -L_i(V^{n+1}),
// solved after each step by restarted GMRES (Sec. 3.2) started from the
// extrapolation 2 v_e^n - v_e^{n-1} once two consecutive solutions are held
// (from v_e^n before that, as the paper does), and the intracellular flux of v_e, L_i(v_e), handed to the next step's
// cell update (which adds it to L_i(V)). L_i is the job's own folded
// operator (the parameter sets' D_l, D_t are the intracellular
// diffusivities); L_ie the same operator folded with D_i + D_e.
#pragma once
#include <cuda_runtime.h>

#include "devtypes.h"

namespace ep {

constexpr int kBidoMaxRestart = 30;   // Krylov dimension limit of one GMRES cycle
constexpr int kBidoThreads = 256;

// Solver counters, written by the solve kernel.
struct BidoStats {
    long long last_iters;    // Arnoldi steps (products with L_ie) of the last solve
    long long total_iters;
    long long solves;
    double last_res;         // ||b - L_ie x|| at the end of the last solve
    double last_bnorm;       // ||b|| of the last solve
    double alg_bytes;        // algorithmic bytes of all solves (every array a phase touches, once)
    double phase_ms[5];      // device time by phase: node values, fluxes, GS pass 2, GS pass 3, updates
    int failed;              // some solve stopped at max_iter without converging
    int timeout;             // a grid barrier of some solve gave up (sticky until v_e is written)
    int hist;                // consecutive solutions held: 0 none, 1 v_e^n, 2 also v_e^{n-1} (in vprev)
    int pad;
};

// Grid barrier state of the cooperative solve kernel, zeroed before every
// launch (a solve whose barrier gave up leaves it inconsistent).
struct BidoSync {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

struct BidoArgs {
    DevJob job;                  // the job's descriptor (topology, L_i coefficients, V, node scratch, step),
                                 // set by launch_bido: the kernel reads it from the constant bank
    const void *wa, *wb, *q;     // L_ie coefficients (layout of DevJob::wa/wb/q)
    const void *wvol;            // V_c / sum V (gauge weights)
    void *ve, *w;                // [ld] each, zero past n_cells
    void *xdiv, *b;              // [n_cells] each
    void *basis;                 // [(restart + 1) * ld], zero past n_cells
    void *vprev;                 // [ld]: the solution before the last one (initial-guess extrapolation)
    long long ld;
    double *part;                // [(kBidoMaxRestart + 1) * grid] block partials
    BidoStats *stats;
    BidoSync *sync;
    double tol, atol;            // stop when ||r|| <= max(tol ||b||, atol sqrt(n_cells))
    long long max_iter;          // Arnoldi steps per solve
    int restart;
    int mode;                    // 0: solve, then L_i(v_e); 1: only L_i(v_e) from the current v_e
    int reorth;                  // 1: Gram-Schmidt twice (CGS2); 0: once (CGS)
    int pad;
    unsigned long long barrier_limit_ns;   // bound of each grid-barrier wait
};

// Grid of the cooperative solve kernel for a job of n_cells: co-resident on
// this device, and no more blocks than give each thread four cells. It
// depends only on the job and the device, so that a job's results do not
// depend on the batch it is stepped in.
int bido_grid(int precision, int sm_count, long long n_cells);

// One solve (mode 0) or flux refresh (mode 1) of one job on stream s: the
// barrier state is zeroed, then one cooperative launch, with dj (the job's
// current descriptor) passed as part of the kernel parameter.
cudaError_t launch_bido(int precision, const BidoArgs &a, const DevJob &dj, int grid, cudaStream_t s);

// out[perm[c]] = src[c] (as double), and the reverse.
cudaError_t launch_field_gather(int precision, const void *src, const int *perm, long long n, double *out,
                                cudaStream_t s);
cudaError_t launch_field_scatter(int precision, const double *in, const int *perm, long long n, void *dst,
                                 cudaStream_t s);

}  // namespace ep
