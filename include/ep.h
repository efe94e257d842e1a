/*
 * ep.h - C ABI of the B300 monodomain finite-volume library.
 *
 * The library advances the operator-split monodomain equation on a
 * tetrahedral cell-centred finite-volume mesh, the method of Del Corso,
 * Verzicco & Viola, "A fast computational model for the electrophysiology of
 * the whole human heart":
 *
 *   dV_c/dt = (1/V_c) sum_{j=1..4} A_fj (D_fj grad v_fj) . n_fj  -  I_ion(V_c, s_c)  -  I_s,c
 *
 * (Eq. 7 divided by chi C_m V_c, with D = M / (chi C_m) in mm^2/ms and the
 * currents in uA/uF), the face gradient built from inverse-distance node
 * values, Gauss-Green cell gradients and the directional-derivative
 * correction of Eq. 8 (Sec. 3.2), the conductivity tensor rotated into the
 * fibre frame (Eqs. 2-3), and the cell state advanced by Rush-Larsen for the
 * gating variables and forward Euler for everything else (Sec. 3.2), with the
 * stimulus of Eq. 4. A 1D vertex-based finite-volume Purkinje graph (Sec. 3.2)
 * couples to the myocardium at junctions (Sec. 3.3).
 *
 * Units everywhere: length mm, time ms, potential mV, current uA/uF,
 * diffusivity mm^2/ms, concentration mM.
 *
 * Conventions common to every entry point
 *   - Return value: EP_OK (0) or one of the negative-free error codes below;
 *     no C++ exception ever crosses this interface. On error the call has no
 *     effect and ep_last_error() describes it.
 *   - Host buffers passed in belong to the caller and are copied before the
 *     call returns; host buffers passed out are written before it returns.
 *   - Device memory belongs to the library. It is obtained through the
 *     context's allocator callbacks (for example a framework's caching
 *     allocator), or from cudaMalloc when none are given, and returned
 *     through them by ep_job_destroy / ep_context_destroy.
 *   - Cell and node arrays passed in or out are in the CALLER's numbering;
 *     the library renumbers internally (reverse Cuthill-McKee) and undoes it.
 *   - Threading: a context and its jobs are used by one host thread at a time.
 *     Device work is enqueued on the context's stream and is asynchronous,
 *     except where an entry point says it synchronises.
 */
#ifndef EP_H
#define EP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
enum {
    EP_OK = 0,
    EP_EINVAL = 1,      /* bad argument (NULL pointer, size mismatch, out-of-range id) */
    EP_ENOMEM = 2,      /* the allocator callback (or cudaMalloc) returned no memory */
    EP_EMESH = 3,       /* degenerate tet, node index out of range, face shared by >2 tets */
    EP_EUNSTABLE = 4,   /* dt above the explicit stability bound of the diffusion operator */
    EP_ENONFINITE = 5,  /* a NaN/Inf was found in the state */
    EP_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
    EP_ECUDA = 7,       /* a CUDA runtime call failed (message in ep_last_error) */
    EP_ESTATE = 8       /* call not valid in the object's current state (e.g. no params set) */
};

/* ---- cell models (Sec. 3.1) ---- */
enum {
    EP_TP06 = 0,        /* ten Tusscher-Panfilov 2006 ventricular myocyte, 19 state variables */
    EP_CRN = 1,         /* Courtemanche-Ramirez-Nattel 1998 atrial myocyte, 21 state variables */
    EP_STEWART = 2      /* Stewart et al. 2009 Purkinje cell, 20 state variables */
};
#define EP_N_MODELS 3

/* ---- arithmetic of a job ---- */
enum {
    EP_FP32_MIXED = 0,  /* FP32 gates, currents, V and diffusion; [Na]i, [K]i and the
                           SR calcium accumulated as two-float compensated sums */
    EP_FP64_PLAIN = 1   /* everything in FP64 */
};

/* ---- time integration of the non-gating variables (V, concentrations) ---- */
enum {
    EP_INTEGRATOR_FE = 0,  /* forward Euler (Sec. 3.2) */
    EP_INTEGRATOR_AB2 = 1  /* second-order Adams-Bashforth (Sec. 4); the first step after
                              ep_params_set, ep_write_state or ep_set_step_index is forward
                              Euler. The conduction graph's nodes stay forward Euler. */
};

/* ---- Purkinje-muscle junction coupling (Sec. 3.3) ---- */
enum {
    EP_PMJ_RESISTIVE = 0, /* current (V_p - V_m)/R into both sides, scaled by each side's capacitance */
    EP_PMJ_TRIGGERED = 1, /* threshold crossing at one side stimulates the other after a delay */
    EP_PMJ_CELL = 2       /* a triggered communication node between two cells (the 2D shell and the
                             3D myocardium): junction_node holds the source cell */
};

#define EP_MAX_PARAM_SETS 16
#define EP_MAX_STIMULI 8
#define EP_VAR_V 0        /* variable 0 of every model is the transmembrane potential */

typedef struct ep_context ep_context;
typedef struct ep_job ep_job;
typedef struct ep_plan ep_plan;

/* Device allocator callbacks. alloc returns a device pointer aligned to at
 * least 256 bytes, or NULL when out of memory; free releases it. */
typedef void *(*ep_alloc_fn)(size_t bytes, void *user);
typedef void (*ep_free_fn)(void *ptr, size_t bytes, void *user);

/* Mesh of one job. xyz: 3*n_nodes doubles (mm), node k at xyz[3k..3k+2].
 * tet: 4*n_cells node indices; either orientation is accepted (the library
 * orders each tet positively). tri: 3*n_tris node indices of the 2D
 * Purkinje shell's triangles (Sec. 2: a surface medium, discretised by the
 * same cell-centred scheme with edges as faces), or n_tris = 0. The job's
 * cells are the n_cells tets followed by the n_tris triangles; the per-cell
 * arrays below and every state / activation output cover all of them in
 * that order. Tets and triangles share no face (they exchange current only
 * through conduction-graph junctions). cell_model: EP_TP06 / EP_CRN /
 * EP_STEWART per cell, or NULL for all EP_TP06. param_set: bytes indexing
 * ep_params.sets, or NULL for all 0. stim_mask: bytes, bit k set =
 * stimulus protocol k covers the cell, or NULL for none. fibre: 3 doubles
 * per cell, the fibre direction (need not be normalised; a triangle's
 * conductivity acts in its plane), or NULL for isotropic tissue with
 * diffusivity D_l. index_width: how the step's gather indices are stored,
 * as 32-bit indices or as 16-bit offsets (bitwise identical results):
 *   - 0 (the default): the cells' indices as 16-bit offsets where the
 *     library's numbering allows it (a cell's neighbours within 32767 cells
 *     of it and the nodes of each run of 256 cells within a window of 65536:
 *     meshes whose reverse Cuthill-McKee bandwidth is below about 3 x 10^4
 *     cells, e.g. the 9.6M-cell wedge), 24 bytes per cell and step fewer;
 *     the node -> cell entries as 32-bit indices;
 *   - 16: also the node -> cell entries as 16-bit offsets where they fit
 *     (the cells of each run of 32 nodes within a window of 65536, which
 *     spans about six RCM levels: smaller meshes), 2 bytes per entry fewer,
 *     though the node pass measured slower than with 32-bit entries;
 *   - 32: every index 32-bit. */
typedef struct {
    int64_t n_nodes;
    const double *xyz;
    int64_t n_cells;
    const int32_t *tet;
    const uint8_t *cell_model;
    const uint8_t *param_set;
    const uint8_t *stim_mask;
    const double *fibre;
    int64_t n_tris;
    const int32_t *tri;
    int32_t index_width;
    int32_t pad;
} ep_mesh_desc;

/* Parameters of one parameter set. variant (TP06 only): 0 epicardial,
 * 1 mid-myocardial (M), 2 endocardial. D_l, D_t: monodomain diffusivity
 * along and across the fibre, mm^2/ms (Eq. 7: D = M/(chi C_m), M the half
 * harmonic mean of the intra- and extracellular conductivities). gks_scale,
 * gkr_scale multiply the maximal I_Ks and I_Kr conductances; K_o is the
 * extracellular potassium concentration (mM). */
typedef struct {
    int32_t variant;
    int32_t reserved;
    double D_l, D_t;
    double gks_scale, gkr_scale;
    double K_o;
} ep_cell_params;

/* Stimulus protocol (Eq. 4): amplitude (uA/uF, negative depolarises, it
 * enters the equation like I_ion), onset, duration, period (ms; period 0 = one
 * pulse). Times are rounded to whole steps: on at step n when
 * n >= round(t_on/dt) and (n - round(t_on/dt)) mod round(period/dt) <
 * round(duration/dt). */
typedef struct {
    double amplitude, t_on, duration, period;
} ep_stimulus;

typedef struct {
    double dt;                          /* time step, ms */
    int32_t precision;                  /* EP_FP32_MIXED or EP_FP64_PLAIN */
    int32_t n_sets;                     /* 1..EP_MAX_PARAM_SETS */
    ep_cell_params sets[EP_MAX_PARAM_SETS];
    int32_t n_stim;                     /* 0..EP_MAX_STIMULI */
    int32_t integrator;                 /* non-gating variables: EP_INTEGRATOR_FE (Sec. 3.2) or
                                           EP_INTEGRATOR_AB2 (Sec. 4); gates are always Rush-Larsen */
    ep_stimulus stim[EP_MAX_STIMULI];
    double threshold;                   /* activation threshold, mV (Sec. 4 uses 0 mV) */
} ep_params;

/* ---------------------------------------------------------------------- */

/* Create a context bound to one CUDA device (the current one) and stream.
 * alloc/free may both be NULL (then cudaMalloc/cudaFree are used); user is
 * passed back to them. cuda_stream is a cudaStream_t (NULL = legacy default
 * stream). *out receives the context. Besides the memory it takes through
 * alloc, the context holds one 4-byte device word of its own (cudaMalloc),
 * where step kernels report bounded waits that gave up. Errors: EP_EINVAL,
 * EP_ECUDA, EP_ENOMEM. */
int ep_context_create(ep_alloc_fn alloc, ep_free_fn free_fn, void *user,
                      void *cuda_stream, ep_context **out);

/* Change the stream later work is enqueued on. */
int ep_context_set_stream(ep_context *ctx, void *cuda_stream);

/* Destroys the context; every job of the context must have been destroyed. */
int ep_context_destroy(ep_context *ctx);

/* Text of the last error on this context (never NULL; "" when none). With a
 * NULL context, the last error of a failed ep_context_create. */
const char *ep_last_error(const ep_context *ctx);

/* Build one job's mesh (Sec. 3.2): validate the tets, order them positively,
 * match faces, renumber cells and nodes in reverse Cuthill-McKee order
 * (grouped by cell model), build the node-to-cell table of the
 * inverse-distance interpolation and upload the topology. Synchronises.
 * Errors: EP_EINVAL, EP_EMESH, EP_ENOMEM, EP_ECUDA. */
int ep_mesh_create(ep_context *ctx, const ep_mesh_desc *desc, ep_job **out);

/* Set (or replace) the job's parameters: precision, dt, parameter sets,
 * stimuli, threshold. Computes in FP64 the geometry, the conductivity
 * tensors (Eqs. 2-3) and the folded per-cell flux coefficients of Eqs. 7-8,
 * rounds them once to the job's precision and uploads them. On the first
 * call (or when the precision changes) it also allocates the state and sets
 * it to each model's published resting state, the activation times to +inf
 * and the step counter to 0. Rejects a dt at or above the explicit stability
 * bound of the diffusion operator with EP_EUNSTABLE. Synchronises. */
int ep_params_set(ep_job *job, const ep_params *params);

/* Two-phase job creation, for servers that overlap host preparation with
 * device work.
 * ep_plan_create does all host work of ep_mesh_create (+ ep_params_set when
 * params is not NULL): validation, renumbering, face matching, the FP64
 * folding and the stability check. It touches no device, needs no context
 * and may run concurrently in several host threads. Errors as
 * ep_mesh_create / ep_params_set; the message is in ep_last_error(NULL) of
 * the calling thread.
 * ep_plan_bytes: device bytes a job created from the plan will hold (the
 * admission estimate).
 * ep_job_create uploads a plan into a new job of ctx on a private upload
 * stream: it does not wait for work queued on the context's stream.
 * Synchronises that upload stream. The plan may be destroyed afterwards
 * (the job keeps the host mesh it shares with the plan). */
int ep_plan_create(const ep_mesh_desc *desc, const ep_params *params, ep_plan **out);
int64_t ep_plan_bytes(const ep_plan *plan);
/* ep_plan_info: cells, nodes, and the widths (16 or 32 bits) the job's
 * cell gather indices and node -> cell entries will be stored with
 * (ep_mesh_desc.index_width). */
int ep_plan_info(const ep_plan *plan, int64_t *n_cells, int64_t *n_nodes, int32_t *index_width,
                 int32_t *node_index_width);
int ep_plan_destroy(ep_plan *plan);
int ep_job_create(ep_context *ctx, const ep_plan *plan, ep_job **out);

/* Advance n_jobs jobs of one context by n_steps time steps each. All jobs are
 * advanced together: every step is one node-value launch and one fused
 * cell launch per launch group, each covering every resident cell of its
 * jobs. The groups: FP32 jobs that step by forward Euler without the
 * bidomain solve, at most 15 to a group (their descriptors are passed to the
 * kernels as a parameter, read from the constant bank); the other FP32 jobs;
 * the FP64 jobs. A job's results do not depend on its group. Repeated calls
 * with the same job list replay a captured CUDA graph. Asynchronous on the context's stream. Errors: EP_EINVAL (jobs of
 * another context, repeated job, job without params), EP_ECUDA, and
 * EP_ETIMEOUT when a staged cell kernel (launch-shape variants 6 and 7) of an
 * earlier call gave up its bounded wait for a tile's copies: that call's
 * error word is read back asynchronously after it, so the error surfaces at
 * a later ep_step or ep_check_finite. The state of every job stepped since
 * the failed step is then undefined; restore the jobs from a checkpoint
 * (ep_write_state, ep_set_step_index) and call ep_clear_error. */
int ep_step(ep_job *const *jobs, int32_t n_jobs, int64_t n_steps);

/* Copy variable var of cell model `model` to host_out (n = number of cells,
 * caller's order). Cells of another model receive NaN, except for
 * EP_VAR_V, which every cell has. Synchronises the context's stream. */
int ep_read_state(ep_job *job, int32_t model, int32_t var, double *host_out, int64_t n);

/* Overwrite variable var of cells of `model` from host_in (n cells, caller's
 * order; entries of cells of other models are ignored, except for EP_VAR_V).
 * With ep_read_state and ep_set_step_index this checkpoints and resumes a job
 * exactly. Synchronises. */
int ep_write_state(ep_job *job, int32_t model, int32_t var, const double *host_in, int64_t n);

/* The same transfers in FP32, for an EP_FP32_MIXED job: V and the variables
 * such a job stores in FP32 (ep_model_var_compensated() == 0) are read and
 * written exactly, with half the bytes of ep_read_state / ep_write_state
 * (a checkpoint of the job's compute-type state, or its upload from a
 * caller that holds it in FP32). Errors: EP_EINVAL for an EP_FP64_PLAIN job,
 * and for a variable stored as a compensated sum ([Na]i, [K]i, the SR
 * calcium), whose value needs FP64: transfer those with ep_read_state /
 * ep_write_state. Synchronise. */
int ep_read_state_f32(ep_job *job, int32_t model, int32_t var, float *host_out, int64_t n);
int ep_write_state_f32(ep_job *job, int32_t model, int32_t var, const float *host_in, int64_t n);

/* Activation times (ms): the first upward crossing of the threshold,
 * t^n + dt (theta - V^n)/(V^{n+1} - V^n) (Sec. 4); +inf where the cell has not
 * activated. n = number of cells, caller's order. Synchronises. */
int ep_activation_times(ep_job *job, double *host_out, int64_t n);
/* The same as FP32 values, for an EP_FP32_MIXED job (the times it stores,
 * exactly; EP_EINVAL for an EP_FP64_PLAIN job). */
int ep_activation_times_f32(ep_job *job, float *host_out, int64_t n);

/* Reset activation times to +inf (a new beat). Asynchronous. */
int ep_reset_activation(ep_job *job);

/* Steps taken so far (synchronises) / set the step counter (t^n = n dt). */
int ep_step_index(ep_job *job, int64_t *out);
int ep_set_step_index(ep_job *job, int64_t n);

/* Scan the job's state for NaN/Inf on the device. Returns EP_OK,
 * EP_ENONFINITE, or EP_ETIMEOUT if a step kernel of the context gave up a
 * bounded wait (the staged cell kernel waits at most 1 s for the bulk copies
 * of a tile; the state is then not valid). Synchronises. */
int ep_check_finite(ep_job *job);

/* Clear the context's record of a step kernel's bounded wait that gave up
 * (after the jobs were restored from a checkpoint): later ep_step calls run
 * again. Synchronises the context's stream. */
int ep_clear_error(ep_context *ctx);

/* Job information: cells, nodes, interior faces, device bytes held, and
 * the widths (16 or 32 bits) of its stored cell gather indices and node ->
 * cell entries (the node-value pass's table). */
int ep_job_info(const ep_job *job, int64_t *n_cells, int64_t *n_nodes,
                int64_t *n_interior_faces, int64_t *device_bytes, int32_t *index_width,
                int32_t *node_index_width);

/* Device bytes a job of this size would hold (planner estimate used for
 * admission by free memory). */
int64_t ep_estimate_bytes(int64_t n_cells, int64_t n_nodes, int32_t precision);

/* Release the job's device memory (after its queued work completes). */
int ep_job_destroy(ep_job *job);

/* Profiling hook: advance the jobs by n_steps with direct launches (no
 * graph), recording CUDA events on the context's stream around each launch,
 * and return the mean device time per step of the node-value kernel and of
 * the fused cell kernel (ms, summed over the jobs' launch groups).
 * The elliptic solves of bidomain jobs run after each step, untimed.
 * Synchronises. The results equal those of ep_step. */
int ep_time_kernels(ep_job *const *jobs, int32_t n_jobs, int64_t n_steps, double *node_ms, double *cell_ms);

/* Autotuner of the step's launch shape. Variants 0-5, 10 and 11: threads
 * per block and resident blocks per SM of the cell kernel, after its own
 * node-value launch (256 x 2, 256 x 3, 128 x 4, 128 x 5, 128 x 6, 64 x 12,
 * 128 x 7, 128 x 8; the block count caps the registers per thread); an
 * FP32 launch group of forward-Euler monodomain jobs (at most 15, see
 * ep_step) runs these shapes, and its node-value launch, with the jobs'
 * descriptors passed as a kernel parameter, read from the constant bank;
 * variants 6 and 7: the staged FP32 cell kernel, whose streamed
 * inputs are brought into shared memory by bulk asynchronous copies,
 * double-buffered (6: all of them, two blocks per SM; 7: indices,
 * coefficients, V and bytes, three blocks per SM), for jobs with 32-bit
 * gather indices (FP64, AB2 and 16-bit-index batches run variant 0 for
 * them); variants 8 and 9: the fused step, node values and cell update of
 * every job in ONE persistent launch (128 threads x 6 blocks per SM, 256 x
 * 3), node tiles and cell tiles taken in dependency order with bounded
 * waits on per-tile ready flags (a wait that gives up sets the context's
 * error word, reported as EP_ETIMEOUT by ep_step and ep_check_finite).
 * Advances the jobs by 12 * steps_per_variant real time steps, timing each
 * variant's whole step (node values, conduction graphs, cell update) with
 * CUDA events, and keeps the fastest variant per precision for every later
 * ep_step of the context. The variants compute the same arithmetic; TP06
 * and Stewart cells agree bitwise across all of them, Courtemanche cells can
 * differ in the last bits between the register-limited shapes and the
 * others. chosen[2] (may be NULL) receives the variant picked for
 * EP_FP32_MIXED and EP_FP64_PLAIN (-1 if no job of that precision);
 * variant_ms[2 * 12] (may be NULL) the mean step time per variant.
 * Synchronises. */
int ep_autotune(ep_job *const *jobs, int32_t n_jobs, int32_t steps_per_variant, int32_t *chosen,
                double *variant_ms);

/* Measured issue rates of the arithmetic pipes the cell step runs on, for
 * the ALU roofs of the cell kernels (the FP64 plain step is bound by the
 * FP64 pipe, the FP32 step by HBM). Each probe fills every SM with
 * independent dependency chains and is timed with CUDA events on the
 * context's stream (best of five, after a warm-up launch). out[3] receives
 * operations per second: out[0] FP32 FMA flops (an FMA counts two),
 * out[1] MUFU ex2 results, out[2] FP64 FMA flops. Takes a few
 * milliseconds, allocates 256 bytes through the context's allocator and
 * synchronises. */
int ep_alu_peaks(ep_context *ctx, double *out);

/* Force the step's launch-shape variant (0..11, see ep_autotune) for one
 * precision. */
int ep_set_cell_variant(ep_context *ctx, int32_t precision, int32_t variant);

/* Host-only inspection of the planner (no device work, no GPU needed): run
 * the mesh ingest and the FP64 coefficient folding of ep_mesh_create +
 * ep_params_set and return the folded operator, so that it can be checked
 * against a face-by-face evaluation of Eqs. 7-8. Output arrays are
 * caller-allocated: cell_order[n_cells] (internal position -> caller cell),
 * tet/opp/nbr/wa/wb/q[4 n_cells] in internal numbering (opp/nbr -1 on the
 * boundary), n2c_ptr[n_nodes + 1], n2c[4 n_cells], nw[4 n_cells] (node ->
 * cell inverse-distance weights). The diffusion term of internal cell c is
 *   sum_k wa[4c+k] vn[tet[4c+k]] + wb[4c+k] vn[opp[4c+k]] + q[4c+k] (V[nbr[4c+k]] - V[c]),
 *   vn[n] = sum_{j in [n2c_ptr[n], n2c_ptr[n+1])} nw[j] V[n2c[j]].
 * *rho_bound receives the Gershgorin bound of the operator's spectral radius.
 * Any output pointer may be NULL. */
int ep_plan_inspect(const ep_mesh_desc *desc, const ep_params *params, int64_t *cell_order, int32_t *tet,
                    int32_t *opp, int32_t *nbr, double *wa, double *wb, double *q, int64_t *n2c_ptr,
                    int32_t *n2c, double *nw, double *rho_bound);

/* Step one job without allocating any device memory. The paper has no
 * counterpart: this entry point is for callers that must not allocate while
 * they step, such as a process whose device memory is entirely reserved by
 * another runtime's pool (a fresh cudaMalloc would fail or fragment it) or a
 * latency-critical loop that may not call cudaMalloc/cudaFree, which can take
 * a global lock or synchronise the device. ep_step, by contrast, builds and
 * caches a batch plan (device job and tile tables) on its first call for a
 * job list, and each job holds its own node-value buffer.
 *
 * The job's state and coefficient arrays (created earlier through the
 * context's allocator) are the inputs and outputs. Everything else the step
 * needs -- a copy of the job's descriptor, its tile tables, a ticket counter
 * and the node values -- lives in one static device array of the library
 * (about 18.3 MiB: EP_NOALLOC_MAX_NODES doubles of node values plus the tile
 * tables and the fused step's work list of EP_NOALLOC_MAX_CELLS cells), held
 * by every GPU that loads the library until the process exits; the
 * descriptor, tiles and work list are copied in
 * from host memory on every call. The step then runs the same kernels as
 * ep_step (in the context's current launch shape, no graph replay), so the
 * results equal ep_step's bit for bit.
 *   - Rejects meshes with more than EP_NOALLOC_MAX_NODES nodes or
 *     EP_NOALLOC_MAX_CELLS cells (EP_EINVAL), and jobs with a conduction
 *     graph, bidomain or AB2 (EP_EINVAL: use ep_step).
 *   - The first call in a CUDA context (one per device, unless the caller
 *     re-creates it, e.g. after cudaDeviceReset) looks up the array's device
 *     address with that context current; make that first call before any
 *     stream capture.
 *   - All calls share the array and it keeps the last call's contents (the
 *     ticket is cleared by each call): calls that overlap on the GPU (other
 *     streams, threads or contexts on the same device) race on it;
 *     serialise them.
 * Asynchronous on the context's stream. */
#define EP_NOALLOC_MAX_NODES 2097152
#define EP_NOALLOC_MAX_CELLS 16777216
int ep_step_noalloc(ep_job *job, int64_t n_steps);

/* ---- conduction graph (Purkinje network, 1D bundles) and junctions ---- */

/* A 1D conduction graph attached to a job (Sec. 3.2: vertex-based FV on a
 * graph, several branches allowed at a node). Node i obeys
 *   dV_i/dt = (2 / sum_j L_ij) sum_j D_ij (V_j - V_i) / L_ij - I_ion - I_s - I_junction
 * with L_ij the edge length and D_ij its diffusivity (mm^2/ms). Every node
 * carries the cell model of its parameter set's model (node_model) with the
 * job's parameter sets. The diffusion is subcycled within each step (the
 * reaction frozen at step n) with k = max(1, ceil(dt rho / 1.8)) substeps,
 * rho = max_i 2 sum_j c_ij, c_ij = 2 D_ij / (L_ij sum_k L_ik).
 * Junctions (Sec. 3.3) pair graph node junction_node[j] with myocardial cell
 * junction_cell[j] (caller numbering):
 *   EP_PMJ_RESISTIVE: g_graph (V_p - V_m) leaves the node and g_cell (V_m - V_p)
 *     leaves the cell, at step n (rates in 1/ms);
 *   EP_PMJ_TRIGGERED: each upward crossing of `threshold` by V_p (time t_p,
 *     interpolated) stimulates every cell within `radius` mm of the junction
 *     cell with `amplitude` over [t_p + delay_ortho, t_p + delay_ortho +
 *     duration); with two_way, crossings by V_m at t_m stimulate the node over
 *     [t_m + delay_anti, ... + duration);
 *   EP_PMJ_CELL: the same with a source cell s = junction_node[j] (caller
 *     cell numbering, e.g. a shell triangle) in place of the node: crossings
 *     by V_s stimulate the cells within `radius` of cell m, and with two_way
 *     crossings by V_m stimulate cell s. A graph may consist of such
 *     junctions alone (n_nodes = 0).
 * Triggered targets are the cells of the junction cell's medium (tets or
 * shell triangles) within `radius` of it.
 * xyz: 3 n_nodes doubles; edges: 2 n_edges node indices; edge_D: per-edge
 * diffusivity or NULL (then params->D); node_model / node_param_set /
 * node_stim_mask: per node or NULL (Stewart / 0 / none); junction_mode: per
 * junction or NULL (all params->default_mode). */
typedef struct {
    int64_t n_nodes;
    const double *xyz;
    int64_t n_edges;
    const int32_t *edges;
    const double *edge_D;
    const uint8_t *node_model;
    const uint8_t *node_param_set;
    const uint8_t *node_stim_mask;
    int64_t n_junctions;
    const int32_t *junction_node;
    const int32_t *junction_cell;
    const uint8_t *junction_mode;
} ep_graph_desc;

typedef struct {
    double D;                         /* default edge diffusivity, mm^2/ms */
    double g_graph, g_cell;           /* resistive junction rates, 1/ms */
    double threshold;                 /* triggered junction threshold, mV (Sec. 3.3: 0 mV) */
    double delay_ortho, delay_anti;   /* ms (Sec. 3.3: 5 ms orthodromic; Sec. 1: 2-3 ms antidromic) */
    double amplitude, duration;       /* triggered stimulus: uA/uF and ms (Sec. 3.3: S_d = 0.5 ms) */
    double radius;                    /* R_S, mm (Sec. 3.3: 0.1 mm Purkinje, 1 mm atria) */
    int32_t two_way;                  /* 1: muscle -> graph triggering too */
    int32_t default_mode;             /* EP_PMJ_RESISTIVE or EP_PMJ_TRIGGERED */
} ep_graph_params;

/* Attach (or replace) the job's conduction graph. The job must have
 * parameters. Graph nodes start at their models' resting states; the graph
 * is rebuilt for a later ep_params_set. Synchronises. Errors: EP_EINVAL
 * (bad index, parameter set, or mode), EP_ESTATE (no parameters). */
int ep_graph_attach(ep_job *job, const ep_graph_desc *desc, const ep_graph_params *params);

/* Graph node state / activation times in the caller's node order (as
 * ep_read_state / ep_write_state / ep_activation_times), and the graph's
 * node count and diffusion substeps per time step. Synchronise. */
int ep_graph_read_state(ep_job *job, int32_t model, int32_t var, double *host_out, int64_t n);
int ep_graph_write_state(ep_job *job, int32_t model, int32_t var, const double *host_in, int64_t n);
int ep_graph_activation_times(ep_job *job, double *host_out, int64_t n);
int ep_graph_info(const ep_job *job, int64_t *n_nodes, int32_t *substeps, int64_t *n_junctions);

/* How a step advances the conduction graphs' diffusion substeps (Sec. 3.2:
 * the vertex-based 1D FV, subcycled for explicit stability):
 * EP_GRAPH_SUBSTEPS_LOCAL (the default) runs all substeps of a step in one
 * launch, each block on a tile of 256 graph nodes and every node within
 * `substeps` hops of it in shared memory (the tile's own values are exact:
 * an error at the rim of the neighbourhood moves one hop per substep);
 * EP_GRAPH_SUBSTEPS_LAUNCHES launches one pass over all graph nodes per
 * substep. Both give bitwise identical results. A batch whose largest
 * neighbourhood does not fit 48 KB of shared memory takes the launches. */
#define EP_GRAPH_SUBSTEPS_LAUNCHES 0
#define EP_GRAPH_SUBSTEPS_LOCAL 1
int ep_set_graph_kernel(ep_context *ctx, int32_t mode);

/* ---- bidomain (Eq. 1, Eqs. 5-6) -------------------------------------------
 * Settings of the elliptic solve (restarted GMRES, Sec. 3.2). A solve stops
 * when ||b - L_ie v_e|| <= max(tol ||b||, atol sqrt(n_cells)) (2-norms over
 * cells, b in mV/ms per cell) or after max_iter Arnoldi steps; the Krylov
 * basis restarts every `restart` steps (1..30) from the true residual;
 * reorth = 1 applies classical Gram-Schmidt twice (CGS2), 0 once (CGS).
 * barrier_limit_s bounds each wait of the solve kernel's grid barriers
 * (seconds; <= 0 takes the default of 2 s): past it the waiting block raises
 * the solve's error flag and every block leaves the kernel at its next
 * barrier (see ep_bidomain_stats). */
typedef struct {
    double tol, atol;
    int32_t restart;
    int32_t reorth;
    int64_t max_iter;
    double barrier_limit_s;
} ep_bidomain_solver;

/* Switch a job to the bidomain model. The parameter sets' (D_l, D_t) become
 * the intracellular diffusivities D_i; De_l[k], De_t[k] (mm^2/ms, k <
 * n_sets = the job's parameter-set count) are the extracellular ones of set
 * k, in the same fibre frame (Eqs. 2-3). Each ep_step then
 *   1. updates V with the intracellular flux of V^n + v_e^n (first line of
 *      Eq. 6), everything else as in the monodomain step;
 *   2. solves the second line of Eq. 6, L_ie(v_e^{n+1}) = -L_i(V^{n+1}), by
 *      restarted GMRES, L_ie being the same finite-volume operator for
 *      D_i + D_e. The solve starts from 2 v_e^n - v_e^{n-1} once two
 *      consecutive solutions are held, else from v_e^n; a v_e written by
 *      ep_bidomain_write_ve counts as one solution;
 *   3. fixes v_e to zero volume-weighted mean (the equation leaves a
 *      constant free under zero-flux boundaries).
 * solver NULL takes the defaults: restart 12, CGS, max_iter 2000, and
 * tol 1e-5, atol 1e-3 mV/ms (FP32 mixed: about the rounding floor of an FP32
 * residual) or tol 1e-11, atol 1e-11 mV/ms (FP64 plain: far above an FP64
 * residual's rounding floor, so that a right-hand side near zero -- a
 * uniform tissue at rest -- still meets the rule).
 * v_e is solved once from the current V before returning. Calling it again
 * replaces the settings; ep_params_set keeps them (and rebuilds the
 * operator). The solve is one cooperative launch per job and step on the
 * context's stream; steps of batches that hold bidomain jobs are not
 * captured in CUDA graphs. Device memory: (restart + 5) values per cell plus
 * the L_ie coefficients. Synchronises. Errors: EP_EINVAL (bad sizes or
 * settings), EP_ESTATE (no parameters), EP_ENOMEM; on error the job is left
 * monodomain. */
int ep_bidomain_enable(ep_job *job, const double *De_l, const double *De_t, int32_t n_sets,
                       const ep_bidomain_solver *solver);

/* Back to the monodomain model (frees the bidomain state). */
int ep_bidomain_disable(ep_job *job);

/* v_e (mV) in the caller's cell order, read or written through host
 * buffers of n = n_cells doubles. A write also recomputes L_i(v_e) for the
 * next step and clears the job's barrier-timeout record (ep_bidomain_stats).
 * Synchronise. Errors: EP_EINVAL (length), EP_ESTATE (not bidomain). */
int ep_bidomain_read_ve(ep_job *job, double *host_out, int64_t n);
int ep_bidomain_write_ve(ep_job *job, const double *host_in, int64_t n);

/* Solver counters of a bidomain job. */
typedef struct {
    int64_t last_iters;    /* Arnoldi steps (products with L_ie) of the last solve */
    int64_t total_iters;   /* ... of all solves */
    int64_t solves;
    double last_res;       /* ||b - L_ie v_e|| at the end of the last solve */
    double last_bnorm;     /* ||b|| of the last solve */
    double alg_bytes;      /* algorithmic device bytes of all solves: each array a phase of
                              the solve touches, counted once per phase */
    double phase_ms[5];    /* device time of all solves by phase: node values, fluxes (with
                              the first Gram-Schmidt dots), second and third Gram-Schmidt
                              passes, updates of v_e and the gauge */
    int32_t failed;        /* some solve stopped at max_iter unconverged */
    int32_t timeout;       /* some solve's grid-barrier wait gave up (sticky, see below) */
} ep_bidomain_stats_t;

/* Fill *out. Synchronises. Returns EP_ETIMEOUT (with *out filled) if a grid
 * barrier wait of some solve since the last ep_bidomain_enable or
 * ep_bidomain_write_ve gave up (ep_bidomain_solver.barrier_limit_s, 2 s by
 * default). Every block of that solve left the kernel; its v_e and the V of
 * the steps after it are undefined. Each later solve re-arms the barrier and
 * runs normally, and other jobs are unaffected. Recovery: restore the job's
 * state and v_e from a checkpoint (ep_write_state, ep_bidomain_write_ve,
 * which clears the record). */
int ep_bidomain_stats(ep_job *job, ep_bidomain_stats_t *out);

/* Number of state variables of a model and the name of each
 * (e.g. "V", "Ca_i", "Na_i", "m"). */
int32_t ep_model_nvar(int32_t model);
const char *ep_model_varname(int32_t model, int32_t var);
/* 1 if variable var of the model is stored as a compensated sum in an
 * EP_FP32_MIXED job (an FP64 value in an EP_FP64_PLAIN one), 0 if it is
 * stored in the job's compute type, -1 for an unknown model or variable. */
int32_t ep_model_var_compensated(int32_t model, int32_t var);

#ifdef __cplusplus
}
#endif
#endif /* EP_H */
