/*
 * FP64 CPU oracle for the monodomain finite-volume step of Del Corso,
 * Verzicco & Viola, "A fast computational model for the electrophysiology of
 * the whole human heart".
 *
 * TEST INFRASTRUCTURE ONLY. This library is the correctness reference the
 * CUDA path is checked against. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product never does. It shares no
 * code, header, table or constant with the CUDA library.
 *
 * It follows the paper's algorithm stage by stage, in plain per-cell loops:
 *   - geometry of the cell-centred tetrahedral FV mesh (Sec. 3.2);
 *   - S1 inverse-distance node values, S2 face values and Gauss-Green cell
 *     gradients, S3 interpolated face gradient with the directional-derivative
 *     correction of Eq. 8, flux A_f (D_f grad v_f).n_f summed over the four
 *     faces, zero on boundary faces (Eq. 7);
 *   - conductivity tensors rotated into the fibre frame (Eqs. 2-3);
 *   - ionic models (ten Tusscher-Panfilov 2006, Courtemanche 1998,
 *     Stewart 2009) advanced by Rush-Larsen for gates and forward Euler for
 *     everything else, all evaluated at (V^n, s^n) (Sec. 3.2);
 *   - the stimulus of Eq. 4 and the activation time (first upward crossing of
 *     a threshold, Sec. 4);
 *   - the 1D vertex-based FV Purkinje graph and its junctions (Sec. 3.2, 3.3);
 *   - the 2D Purkinje shell: triangles with the same cell-centred scheme (Sec. 2, 3.2);
 *   - the bidomain model (Eqs. 1, 5-6): the extracellular potential from the
 *     elliptic equation by restarted GMRES warm-started from the last step.
 *
 * Units: V in mV, t in ms, D in mm^2/ms, currents in uA/uF.
 */
#ifndef EP_ORACLE_H
#define EP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXVAR 24

/* ORC_PASSIVE: a membrane with no ionic current (I_ion = 0, V its only
 * state variable, 0 mV at start); V then moves by diffusion and stimulus
 * alone, which gives closed forms to pin the tissue step against. */
enum { ORC_TP06 = 0, ORC_CRN = 1, ORC_STEWART = 2, ORC_PASSIVE = 3 };

typedef struct {
    int32_t model;      /* ORC_TP06 / ORC_CRN / ORC_STEWART / ORC_PASSIVE */
    int32_t variant;    /* TP06: 0 epi, 1 mid, 2 endo */
    double D_l, D_t;    /* monodomain diffusivity along / across the fibre, mm^2/ms */
    double gks_scale, gkr_scale;
    double K_o;         /* extracellular K+, mM */
} orc_cellparams;

typedef struct {
    double amplitude;   /* uA/uF; negative depolarises (enters like I_ion) */
    double t_on, duration, period;  /* ms; period 0 = single pulse */
} orc_stim;

/* ---- geometry and the diffusion operator (fv3d.c) ---- */
typedef struct orc_mesh orc_mesh;
orc_mesh *orc_mesh_create(int64_t n_nodes, const double *xyz, int64_t n_cells,
                          const int32_t *tet, int *err);
void orc_mesh_destroy(orc_mesh *m);
int64_t orc_mesh_n_boundary_faces(const orc_mesh *m);
void orc_mesh_cell_info(const orc_mesh *m, double *centroid, double *volume,
                        int32_t *neighbour);
void orc_node_values(const orc_mesh *m, const double *v, double *vn);
void orc_cell_gradients(const orc_mesh *m, const double *vn, double *grad);
void orc_diffusion(const orc_mesh *m, const double *D, const double *v, double *out);
void orc_diffusion_twopoint(const orc_mesh *m, const double *D, const double *v, double *out);
void orc_conductivity(const double *fibre, double D_l, double D_t, double *D);

/* ---- cell models (tp06.c, crn.c, stewart.c) ---- */
int orc_model_nvar(int model);
const char *orc_model_varname(int model, int var);
void orc_model_init(const orc_cellparams *p, double *s);
/* Second-order Adams-Bashforth for the non-gating variables (Sec. 4: the
 * alternative to forward Euler the paper tests). h holds ORC_NHIST rates of
 * the previous step: slot 0 the V equation (tissue.c), 1..5 the model's
 * non-gating variables; `on` is 0 on the first step after a (re)start,
 * which is forward Euler and only records the rates. */
#define ORC_NHIST 6
typedef struct {
    double *h;
    int on;
} orc_ab2;

/* The rate a non-gating variable advances with over the step: f (forward
 * Euler, ab NULL or off) or 3/2 f - 1/2 f_prev (AB2); slot k then holds f. */
static inline double orc_rate(orc_ab2 *ab, int k, double f) {
    if (!ab) return f;
    const double g = ab->on ? 1.5 * f - 0.5 * ab->h[k] : f;
    ab->h[k] = f;
    return g;
}

double orc_model_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab);
/* single-cell run: V recorded every record_every steps (n_steps/record_every values) */
void orc_cell_run(const orc_cellparams *p, double dt, int64_t n_steps,
                  const orc_stim *stim, int64_t record_every, double *v_out,
                  double *state_inout, int ab2);

/* ---- the 2D Purkinje shell: triangles in 3D space (fv2d.c) ---- */
typedef struct orc_shell orc_shell;
orc_shell *orc_shell_create(int64_t n_nodes, const double *xyz, int64_t n_cells, const int32_t *tri, int *err);
void orc_shell_destroy(orc_shell *s);
void orc_shell_node_values(const orc_shell *s, const double *v, double *vn);
void orc_shell_gradients(const orc_shell *s, const double *vn, double *grad);
void orc_shell_diffusion(const orc_shell *s, const double *D, const double *v, double *out);
void orc_shell_cell_info(const orc_shell *s, double *centroid, double *area, int32_t *neighbour);

/* ---- tissue simulation (tissue.c) ---- */
typedef struct orc_sim orc_sim;
orc_sim *orc_sim_create(int64_t n_nodes, const double *xyz, int64_t n_cells,
                        const int32_t *tet, const double *fibre,
                        const uint8_t *param_set, const uint8_t *stim_mask,
                        int n_sets, const orc_cellparams *sets,
                        int n_stim, const orc_stim *stim,
                        double dt, double threshold, int *err);
orc_sim *orc_sim_create2(int64_t n_nodes, const double *xyz, int64_t n_tets,
                         const int32_t *tet, int64_t n_tris, const int32_t *tri, const double *fibre,
                         const uint8_t *param_set, const uint8_t *stim_mask,
                         int n_sets, const orc_cellparams *sets,
                         int n_stim, const orc_stim *stim,
                         double dt, double threshold, int *err);
void orc_sim_destroy(orc_sim *s);
int orc_set_threads(int n);
void orc_sim_run(orc_sim *s, int64_t n_steps);
int64_t orc_sim_step_index(const orc_sim *s);
void orc_sim_get_var(const orc_sim *s, int var, double *out);
void orc_sim_set_var(orc_sim *s, int var, const double *in);
void orc_sim_get_act(const orc_sim *s, double *out);
void orc_sim_set_step_index(orc_sim *s, int64_t n);
int orc_sim_set_integrator(orc_sim *s, int integrator);
void orc_sim_diffusion(const orc_sim *s, const double *v, double *out);
const orc_mesh *orc_sim_mesh(const orc_sim *s);
/* bidomain (tissue.c): extracellular diffusivities per parameter set, the
 * GMRES stopping rule; v_e state, solver statistics, the elliptic operator */
int orc_sim_set_bidomain(orc_sim *s, const double *De_l, const double *De_t, double tol, int restart,
                         int64_t max_iter);
void orc_sim_get_ve(const orc_sim *s, double *out);
void orc_sim_set_ve(orc_sim *s, const double *in);
void orc_sim_bidomain_stats(const orc_sim *s, double *stats);
void orc_sim_bidomain_operator(const orc_sim *s, const double *x, double *out);
int orc_stim_active(const orc_stim *st, double dt, int64_t n);

/* ---- conduction graph and junctions (purkinje.c) ---- */
/* junction modes: a graph node and a cell, by resistance or by a triggered
 * stimulus; or a communication node between two cells (jnode is then the
 * source cell, e.g. a Purkinje-shell triangle, jcell the target myocardial
 * cell), triggered like ORC_JUNC_TRIGGERED */
enum { ORC_JUNC_RESISTIVE = 0, ORC_JUNC_TRIGGERED = 1, ORC_JUNC_CELL = 2 };
typedef struct {
    double D;                        /* default edge diffusivity, mm^2/ms */
    double g_graph, g_cell;          /* resistive coupling rates, 1/ms */
    double threshold;                /* triggered: crossing threshold, mV */
    double delay_ortho, delay_anti;  /* ms */
    double amplitude, duration;      /* triggered stimulus, uA/uF and ms */
    double radius;                   /* triggered: target cells within this distance, mm */
    int32_t two_way, pad;
    double act_threshold;            /* activation threshold of graph nodes (set by the sim) */
} orc_graph_params;
typedef struct orc_graph orc_graph;
orc_graph *orc_graph_build(int64_t n, const double *xyz, int64_t n_edges, const int32_t *edges,
                           const double *edge_D, const uint8_t *pset, const uint8_t *smask,
                           int n_sets, const orc_cellparams *sets, double dt,
                           int64_t n_junc, const int32_t *jnode, const int32_t *jcell,
                           const uint8_t *jmode, const orc_graph_params *p,
                           int64_t n_cells, const double *cell_centroid, int64_t n_tets, int *err);
void orc_graph_free(orc_graph *g);
int orc_graph_substeps(const orc_graph *g);
int64_t orc_graph_n(const orc_graph *g);
double *orc_graph_state(orc_graph *g);
double *orc_graph_act(orc_graph *g);
void orc_graph_cell_terms(const orc_graph *g, const double *V, double t, double *i_extra, double *s_extra);
void orc_graph_step(orc_graph *g, const double *V3, double t, double dt, int64_t n_step,
                    const orc_cellparams *sets, const orc_stim *stim, int n_stim);
void orc_graph_triggers(orc_graph *g, const double *V3_old, const double *V3_new, const double *Vg_old,
                        double t, double dt);

int orc_sim_attach_graph(orc_sim *s, int64_t n, const double *xyz, int64_t n_edges, const int32_t *edges,
                         const double *edge_D, const uint8_t *pset, const uint8_t *smask,
                         int64_t n_junc, const int32_t *jnode, const int32_t *jcell, const uint8_t *jmode,
                         const orc_graph_params *p);
int orc_sim_graph_substeps(const orc_sim *s);
void orc_graph_laplacian(const orc_graph *g, const double *W, double *out);
void orc_sim_graph_laplacian(const orc_sim *s, const double *W, double *out);
void orc_sim_graph_get_var(const orc_sim *s, int var, double *out);
void orc_sim_graph_set_var(orc_sim *s, int var, const double *in);
void orc_sim_graph_get_act(const orc_sim *s, double *out);

#ifdef __cplusplus
}
#endif
#endif
