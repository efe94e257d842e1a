// Launch wrappers of the device kernels (kernels.cu), callable from host C++.
#pragma once
#include <cuda_runtime.h>

#include "devtypes.h"

namespace ep {

// Descriptors of a small FP32 batch passed as a kernel parameter (constant
// bank; the parameter space holds 32 KB, room for kParamJobs descriptors):
// the kernels read a job's fields -- array bases, region strides, parameter
// sets, stimulus protocols, dt -- from the constant bank, as operands that
// hold no registers, instead of loading them into registers through L1 / L2
// from the job table. The tiles of job j are cell tiles [cell_begin[j],
// cell_begin[j + 1]) and node tiles [node_begin[j], node_begin[j + 1]) of
// the launch (a batch's tiles are grouped by job, in job order).
constexpr int kParamJobs = 15;
template <int K>
struct JobTab {
    int n_jobs;
    int cell_begin[K + 1];
    int node_begin[K + 1];
    DevJob j[K];
};

struct StepLaunch {
    const DevJob *jobs;        // device job table
    int n_jobs;
    const Tile *node_tiles;
    int n_node_tiles;
    const Tile *cell_tiles;
    int n_cell_tiles;
    unsigned *done;            // device counter used to advance the step counters
    int node_grid, cell_grid;  // persistent grid sizes
    int cell_grid0;            // the grid of variant 0 (what staged variants fall back to)
    int cell_variant;          // launch shape of the cell kernel (EP_CELL_VARIANTS)
    const Tile *graph_tiles;   // conduction-graph nodes of all jobs (none: n_graph_tiles = 0)
    int n_graph_tiles;
    int graph_grid;
    int graph_substeps;        // largest substep count of the jobs' graphs
    const Tile *graph_sub_tiles;   // graph tiles with the job-local tile index in Tile::model
    int graph_local;           // all substeps in one launch per tile (graph_substeps_kernel)
    int graph_lmax;            // largest local slot count over the jobs' graph tiles
    int bido;                  // some job is bidomain (cell kernel adds DevJob::xdiv)
    int ab2;                   // some job integrates by AB2 (cell kernel keeps rate histories)
    int idx16;                 // some job stores 16-bit gather indices (the staged variants need 32-bit)
    int sm_count;              // SMs of the device (grid of the one-job cell kernel, sized by its own occupancy)
    int node_form;             // node -> cell entries of the batch: 0 all 32-bit, 1 all 16-bit, 2 mixed
    int models;                // cell models of the batch's cells, bit m for model m
    unsigned *err;             // device error word of the context (bounded waits that gave up)
    const JobTab<1> *tab1;     // host copies of the descriptors of a batch of one job,
    const JobTab<kParamJobs> *tabk;   // or of up to kParamJobs jobs (else NULL)
    const Work *work;          // fused variants: node and cell tiles in dependency order
    int n_work;
    unsigned *head;            // fused variants: next work item (device counter)
};

// Launch shapes of the cell kernel: (index, threads per block, minimum
// resident blocks per SM, which caps the registers per thread). Variant 0 is
// the default before autotuning. An FP32 batch of at most kParamJobs jobs
// (forward Euler, monodomain) runs these shapes as cell_kernel_tab, the
// jobs' descriptors a kernel parameter.
#define EP_CELL_VARIANTS(X) \
    X(0, 256, 2)            \
    X(1, 256, 3)            \
    X(2, 128, 4)            \
    X(3, 128, 5)            \
    X(4, 128, 6)            \
    X(5, 64, 12)            \
    X(10, 128, 7)           \
    X(11, 128, 8)
// Variants 6 and 7: cell_kernel_staged (FP32 forward Euler, 32-bit indices,
// 256 threads; streamed inputs staged by bulk copies: 6 everything, two
// blocks per SM; 7 indices / coefficients / V / bytes, three blocks per SM);
// for FP64, AB2 or 16-bit-index batches they run variant 0.
// Variants 8 and 9: the fused step (fused_kernel: node tiles and cell tiles
// of every job in one persistent launch, in dependency order; 128 threads x
// 6 blocks per SM and 256 x 3).
#define EP_FUSED_VARIANTS(X) \
    X(8, 128, 6)             \
    X(9, 256, 3)
constexpr int kNumCellVariants = 12;
constexpr int kStagedVariant = 6;
constexpr int kFusedVariant = 8;
constexpr bool is_staged_variant(int v) { return v >= kStagedVariant && v < kFusedVariant; }
constexpr bool is_fused_variant(int v) { return v >= kFusedVariant && v < kFusedVariant + 2; }
constexpr int kFusedLookahead = 8192;   // cell tiles whose node tiles are queued ahead of them
constexpr int kFusedChunk = 8;          // node tiles per completion counter of the fused step
int cell_variant_threads(int variant);

// One time step of every job in the table: node values, the conduction
// graphs (reaction, then the diffusion substeps), then the fused diffusion +
// cell-model + activation update.
cudaError_t launch_step(int precision, const StepLaunch &L, cudaStream_t s);

// Graph substep modes: one launch per substep over all graph nodes, or all
// substeps of a step in one launch, each tile on its own nodes and their
// neighbourhood in shared memory (when three arrays of graph_lmax values fit
// kGraphLocalMaxBytes; else the batch takes one launch per substep).
constexpr size_t kGraphLocalMaxBytes = 48 * 1024;

// Set the state of every cell to its model's resting state, activation
// times to +inf (job given by a device pointer to its DevJob).
cudaError_t launch_init(int precision, const DevJob *job, long long n_cells, cudaStream_t s);

// The parts of launch_step, separately (for timing): node values, the
// conduction graphs (no launch when no job has one), the cell update. With a
// fused variant the node part is empty and the cell part is the fused launch.
cudaError_t launch_node(int precision, const StepLaunch &L, cudaStream_t s);
cudaError_t launch_graph(int precision, const StepLaunch &L, cudaStream_t s);
cudaError_t launch_cell(int precision, const StepLaunch &L, cudaStream_t s);

// Copy variable `var` of `model` (all cells for var 0 = V) into out[n_cells]
// in the caller's cell order (internal cell c -> out[perm[c]]; cells of other
// models get NaN), and the reverse.
cudaError_t launch_gather(int precision, const DevJob *job, const int *perm, long long n_cells, int model, int var,
                          double *out, cudaStream_t s);
cudaError_t launch_scatter(int precision, const DevJob *job, const int *perm, long long n_cells, int model, int var,
                           const double *in, cudaStream_t s);
cudaError_t launch_gather_act(int precision, const DevJob *job, const int *perm, long long n_cells, double *out,
                              cudaStream_t s);
cudaError_t launch_reset_act(int precision, const DevJob *job, long long n_cells, cudaStream_t s);
// The same transfers of an FP32 job in FP32 (variables stored in FP32 and
// V; the activation times): write = 0 gathers into buf, 1 scatters from it.
cudaError_t launch_transfer_f32(const DevJob *job, const int *perm, long long n_cells, int model, int var,
                                float *buf, int write, cudaStream_t s);
cudaError_t launch_gather_act_f32(const DevJob *job, const int *perm, long long n_cells, float *out, cudaStream_t s);

// Count non-finite values of the job's state into *count (device int).
cudaError_t launch_check_finite(int precision, const DevJob *job, long long n_cells, unsigned *count,
                                cudaStream_t s);


// Pipe issue-rate probe (peaks.cu): kind 0 FP32 FMA, 1 MUFU ex2, 2 FP64
// FMA. *ops receives the operations (flops for FMA kinds) of the launch.
cudaError_t launch_alu_probe(int kind, int blocks, int iters, double *sink, cudaStream_t s, double *ops);
int alu_probe_threads();

// Step one job n_steps times like launch_step, with its descriptor, tile
// tables, work list (fused variants), counters and node values in a static
// device array instead of allocated memory (at most EP_NOALLOC_MAX_NODES
// nodes and EP_NOALLOC_MAX_CELLS cells). job, node_tiles, cell_tiles and
// work are host copies (tiles of job 0).
cudaError_t launch_step_noalloc(int precision, const DevJob &job, const Tile *node_tiles, int n_node_tiles,
                                const Tile *cell_tiles, int n_cell_tiles, const Work *work, int n_work,
                                int cell_variant, int sm_count, unsigned *err, long long n_steps, cudaStream_t s);

// The two-launch cell kernel shapes of the plain FP64 step (kernels_f64.cu),
// and of a small FP32 batch whose descriptors are a kernel parameter
// (kernels_tab.cu: tab_eligible says whether a launch qualifies; then its
// node kernel too).
cudaError_t launch_cell_plain_f64(const StepLaunch &L, cudaStream_t s);
int cell_blocks_plain_f64(int variant);
bool tab_eligible(const StepLaunch &L);
cudaError_t launch_cell_tab(const StepLaunch &L, cudaStream_t s);
cudaError_t launch_node_tab(const StepLaunch &L, cudaStream_t s);

// Kernel attributes for sizing persistent grids.
int cell_blocks_per_sm(int precision, int variant);
int node_blocks_per_sm(int precision);

}  // namespace ep
