// Plain-data structures shared by the host runtime and the kernels: one
// DevJob per resident job (the job table of the batched launch) and the tile
// tables that map thread blocks onto cells and nodes.
#pragma once
#include <cstdint>
#include <vector_types.h>

#include "../../include/ep.h"

namespace ep {

// Stimulus protocol in whole steps (Eq. 4).
struct DevStim {
    double amp;
    long long n_on, n_dur, n_per;
    float amp_f;
    int pad;
};

// Per-set parameters, in FP64 for the plain path and rounded once to FP32
// for the mixed path (so the FP32 kernel does no FP64 conversions).
struct DevParams {
    int variant;
    int pad;
    double gks_scale, gkr_scale, K_o, sqrt_Ko;   // sqrt_Ko = sqrt(K_o / 5.4)
    float gks_f, gkr_f, Ko_f, sqrt_Ko_f;
};

// State of the cells of one cell model inside a job: n_r arrays of the
// job's compute type (float or double) and, in a second allocation, n_a
// arrays of 8-byte accumulators: FP64 values in the plain path, two-float
// compensated sums (hi, lo) in the mixed path. Variable v of local cell i is
// r[v * stride + i] (and a[v * stride + i]).
struct DevRegion {
    void *r;
    double *a;
    void *h;              // AB2 rate history, kHistSlots arrays of the compute type (NULL: forward Euler)
    long long stride;
    long long off;   // first cell of the region in the job's numbering
    long long n;
};

// Conduction graph of a job (n_nodes == 0: none). Node potentials are
// double-buffered by the job's step parity like the cells' V.
struct DevGraph {
    long long n_nodes;
    void *V[2];
    void *W[2];                 // substep buffers
    void *itot;                 // reaction current frozen over the step's substeps
    void *act;
    const int *row, *col;       // neighbours (CSR)
    const void *coef;           // c_ij
    const uint8_t *pset, *smask;
    DevRegion reg[EP_N_MODELS];
    int substeps;
    int n_junc;
    const int *jnode, *jcell;
    const uint8_t *jmode;
    double *t_graph, *t_cell;   // last upward threshold crossing of each junction's two sides
    const int *node_junc_ptr, *node_junc;
    const int *tgt_cell, *tgt_junc;
    int n_tgt;
    int two_way;
    int cell_nodes;             // some junction is a cell-to-cell communication node
    // local tables of the one-launch substeps (graph_substeps_kernel): graph tile t
    // works on local slots [lt_ptr[t], lt_ptr[t+1]) -- its own nodes first, then every
    // node within `substeps` hops -- slot = (graph node, offset of its neighbours'
    // local indices in lcol, -1 for a neighbour outside the tile's set)
    const int *lt_ptr;
    const int2 *lslot;
    const int *lcol;
    int lmax;                   // largest slot count of a tile
    int pad_g;
    double g_graph, g_cell, threshold, delay_ortho, delay_anti, amplitude, duration, h;
    float g_graph_f, g_cell_f, amplitude_f, h_f;
};

struct DevJob {
    // Gather indices of the step: the cells' (idx16 selects the form) and the
    // node -> cell entries (col16 selects), each as 32-bit indices or 16-bit offsets.
    const int4 *nodes_a;      // the cell's 4 vertices
    const int4 *nodes_b;      // vertex of the neighbour opposite each face (own vertex 0 on the boundary)
    const int4 *nbr;          // neighbour across each face (the cell itself on the boundary)
    const uint4 *cidx16;      // per cell 8 x u16: nodes_a then nodes_b, from nbase[c >> 8]
    const uint2 *nbr16;       // per cell 4 x s16: nbr relative to the cell
    const int *nbase;         // per run of 256 cells
    const int *ncol;          // sliced-ELL node -> cell entries
    const unsigned short *ncol16;  // the same relative to cbase[slice]
    const int *cbase;         // per slice of 32 nodes
    int idx16, col16;
    const void *wa, *wb, *q;  // float4 or double4 per cell (folded Eqs. 7-8 coefficients / V_c)
    const uint8_t *pset;
    const uint8_t *smask;
    void *V[2];               // double-buffered transmembrane potential
    void *vn;                 // node values (scratch of the step)
    void *act;                // activation times
    const long long *slice_ptr;  // sliced-ELL node -> cell table (entries: ncol / ncol16, nw)
    const void *nw;
    long long n_cells, n_nodes;
    DevRegion reg[EP_N_MODELS];
    DevParams params[EP_MAX_PARAM_SETS];
    DevStim stim[EP_MAX_STIMULI];
    int n_stim;
    int precision;
    double dt, threshold;
    float dt_f, threshold_f;
    long long *step;          // steps taken (device counter)
    unsigned *gen;            // fused launches taken (device counter)
    unsigned *ntflag;         // per chunk of node tiles: node tiles completed over all fused launches
    DevGraph g;
    const void *xdiv;         // bidomain: intracellular flux of v_e, added to the diffusion term (else NULL)
    int integrator;           // EP_INTEGRATOR_FE or EP_INTEGRATOR_AB2 (non-gating variables)
    int pad2;
    long long ab2_from;       // AB2: steps n > ab2_from use the history (the step ab2_from is forward Euler)
};

// A tile is a run of consecutive cells (or nodes) of one job and one model.
struct Tile {
    int job;
    int model;
    int start;
    int count;
};

// Work item of the fused step kernel: a node tile (tile < 0: node tile
// -1 - tile of the launch's node tiles) or a cell tile (tile >= 0) with the
// range [dep_lo, dep_hi] of its job's node tiles (local indices, node >> 8)
// whose values it gathers.
struct Work {
    int tile;
    int dep_lo, dep_hi;
    int pad;
};

constexpr int kCellThreads = 256;
constexpr int kHistSlots = 6;              // AB2 rate history per cell: V and five non-gating variables
constexpr int kGraphThreads = 256;
constexpr unsigned kJunctionFlag = 0x80;   // set in a cell's parameter-set byte when a junction touches it
constexpr int kJunctionSource = 1 << 30;   // in DevGraph::tgt_junc: the cell is the source of a cell-to-cell node
constexpr int kNodeThreads = 256;

}  // namespace ep
