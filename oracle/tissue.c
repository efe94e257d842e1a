/*
 * Oracle (test infrastructure only): the operator-split monodomain time step
 * on the tetrahedral mesh, and the single-cell driver.
 *
 * One step from t^n = n dt (Sec. 3.2, Eq. 7 divided by chi C_m V_c):
 *   diff_c   = (1/V_c) sum_j A_fj (D_fj grad v_fj) . n_fj        (fv3d.c)
 *   I_s,c    = sum of the amplitudes of the stimulus protocols (Eq. 4) that
 *              cover cell c and are on at step n
 *   s^{n+1}  = cell-model update at (V^n, s^n)  (RL gates, FE the rest)
 *   V^{n+1}  = V^n + dt (diff_c - I_ion(V^n, s^n) - I_s,c)
 *   activation time: at the first step with V^n < theta <= V^{n+1},
 *              t_act = t^n + dt (theta - V^n) / (V^{n+1} - V^n)
 * With a conduction graph attached (purkinje.c), the junction terms at step
 * n enter the cells' update (a resistive current beside the diffusion term,
 * a triggered stimulus beside I_s), then the graph advances from its own
 * (V^n, s^n) and the 3D V^n, then junction crossings are recorded.
 *
 * A stimulus protocol is on at step n when n >= n_on and
 * (n - n_on) mod n_period < n_dur (single pulse: n < n_on + n_dur), with
 * n_on, n_dur, n_period the onset, duration and period rounded to whole
 * steps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

/* Thread count of the OpenMP loops of later calls from this thread (n <= 0
 * leaves it); returns the count in effect before. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    const int prev = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return prev;
#else
    (void)n;
    return 1;
#endif
}

int orc_tp06_nvar(void);
const char *orc_tp06_varname(int v);
void orc_tp06_init(int variant, double *s);
double orc_tp06_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab);
int orc_crn_nvar(void);
const char *orc_crn_varname(int v);
void orc_crn_init(double *s);
double orc_crn_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab);
int orc_stewart_nvar(void);
const char *orc_stewart_varname(int v);
void orc_stewart_init(double *s);
double orc_stewart_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab);

int orc_model_nvar(int model) {
    switch (model) {
    case ORC_TP06: return orc_tp06_nvar();
    case ORC_CRN: return orc_crn_nvar();
    case ORC_STEWART: return orc_stewart_nvar();
    case ORC_PASSIVE: return 1;
    }
    return 0;
}

const char *orc_model_varname(int model, int var) {
    switch (model) {
    case ORC_TP06: return orc_tp06_varname(var);
    case ORC_CRN: return orc_crn_varname(var);
    case ORC_STEWART: return orc_stewart_varname(var);
    case ORC_PASSIVE: return var == 0 ? "V" : 0;
    }
    return 0;
}

void orc_model_init(const orc_cellparams *p, double *s) {
    for (int k = 0; k < ORC_MAXVAR; ++k) s[k] = 0.0;
    switch (p->model) {
    case ORC_TP06: orc_tp06_init(p->variant, s); break;
    case ORC_CRN: orc_crn_init(s); break;
    case ORC_STEWART: orc_stewart_init(s); break;
    }
}

/* Advances every state variable except V (index 0); returns I_ion(V^n, s^n)
 * (zero for the passive membrane, which has no other state). */
double orc_model_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab) {
    switch (p->model) {
    case ORC_TP06: return orc_tp06_step(s, dt, i_stim, p, ab);
    case ORC_CRN: return orc_crn_step(s, dt, i_stim, p, ab);
    case ORC_STEWART: return orc_stewart_step(s, dt, i_stim, p, ab);
    }
    return 0.0;
}

int orc_stim_active(const orc_stim *st, double dt, int64_t n) {
    int64_t n_on = llround(st->t_on / dt);
    int64_t n_dur = llround(st->duration / dt);
    int64_t n_per = llround(st->period / dt);
    if (n < n_on) return 0;
    if (n_per <= 0) return n < n_on + n_dur;
    return ((n - n_on) % n_per) < n_dur;
}

void orc_cell_run(const orc_cellparams *p, double dt, int64_t n_steps,
                  const orc_stim *stim, int64_t record_every, double *v_out,
                  double *state_inout, int ab2) {
    double s[ORC_MAXVAR], h[ORC_NHIST] = {0};
    orc_ab2 ab = {h, 0};
    memcpy(s, state_inout, sizeof(s));
    int64_t r = 0;
    for (int64_t n = 0; n < n_steps; ++n) {
        double is = (stim && orc_stim_active(stim, dt, n)) ? stim->amplitude : 0.0;
        double vn = s[0];
        ab.on = n > 0;
        double iion = orc_model_step(s, dt, is, p, ab2 ? &ab : NULL);
        s[0] = vn + dt * orc_rate(ab2 ? &ab : NULL, 0, -iion - is);
        if (record_every > 0 && (n + 1) % record_every == 0) v_out[r++] = s[0];
    }
    memcpy(state_inout, s, sizeof(s));
}

struct orc_sim {
    orc_mesh *m;
    int64_t n_cells;
    uint8_t *pset, *smask;
    int n_sets;
    orc_cellparams sets[256];
    int n_stim;
    orc_stim stim[8];
    double dt, theta;
    int64_t step;
    double *state;   /* [n_cells][ORC_MAXVAR] */
    double *D;       /* [n_cells][9] */
    double *act;
    double *v, *diff;
    orc_graph *g;              /* optional conduction graph */
    double *i_extra, *s_extra, *vg_old, *v_new;
    double *fibre;             /* [n_cells][3] */
    int64_t n_tets;            /* cells [0, n_tets) are tetrahedra, the rest shell triangles */
    orc_shell *shell;
    double *xyz;               /* node coordinates (kept for the shell) */
    int integrator;            /* 0 forward Euler, 1 AB2 for the non-gating variables */
    int64_t ab2_from;          /* step whose rates start the AB2 history (forward Euler there) */
    double *hist;              /* [n_cells][ORC_NHIST] */
    /* bidomain (NULL ve: monodomain) */
    double *ve, *Die, *u, *rhs;
    double gm_tol;
    int gm_restart;
    int64_t gm_max_iter, gm_last_iter, gm_total_iter;
    double gm_last_res;
    int gm_failed;
};

static void bidomain_solve(orc_sim *s);

/* Cells 0 .. n_tets-1 are the tetrahedra, n_tets .. n_tets+n_tris-1 the
 * triangles of the Purkinje shell (fv2d.c); per-cell arrays cover both. The
 * two media share no face: they exchange current only through junctions. */
orc_sim *orc_sim_create2(int64_t n_nodes, const double *xyz, int64_t n_tets,
                         const int32_t *tet, int64_t n_tris, const int32_t *tri, const double *fibre,
                         const uint8_t *param_set, const uint8_t *stim_mask,
                         int n_sets, const orc_cellparams *sets,
                         int n_stim, const orc_stim *stim,
                         double dt, double threshold, int *err) {
    const int64_t n_cells = n_tets + n_tris;
    if (n_sets < 1 || n_sets > 256 || n_stim < 0 || n_stim > 8 || n_cells < 1) { *err = 10; return NULL; }
    for (int64_t c = 0; c < n_cells; ++c)
        if (param_set[c] >= n_sets) { *err = 11; return NULL; }
    orc_mesh *m = NULL;
    if (n_tets > 0) {
        m = orc_mesh_create(n_nodes, xyz, n_tets, tet, err);
        if (!m) return NULL;
    }
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->m = m;
    s->n_tets = n_tets;
    if (n_tris > 0) {
        s->xyz = (double *)malloc(sizeof(double) * 3 * n_nodes);
        memcpy(s->xyz, xyz, sizeof(double) * 3 * n_nodes);
        s->shell = orc_shell_create(n_nodes, s->xyz, n_tris, tri, err);
        if (!s->shell) {
            *err += 20;
            orc_mesh_destroy(m);
            free(s->xyz);
            free(s);
            return NULL;
        }
    }
    s->n_cells = n_cells;
    s->pset = (uint8_t *)malloc(n_cells);
    memcpy(s->pset, param_set, n_cells);
    s->smask = (uint8_t *)malloc(n_cells);
    if (stim_mask) memcpy(s->smask, stim_mask, n_cells);
    else memset(s->smask, 0, n_cells);
    s->n_sets = n_sets;
    memcpy(s->sets, sets, sizeof(orc_cellparams) * n_sets);
    s->n_stim = n_stim;
    if (n_stim) memcpy(s->stim, stim, sizeof(orc_stim) * n_stim);
    s->dt = dt;
    s->theta = threshold;
    s->step = 0;
    s->state = (double *)malloc(sizeof(double) * ORC_MAXVAR * n_cells);
    s->D = (double *)malloc(sizeof(double) * 9 * n_cells);
    s->act = (double *)malloc(sizeof(double) * n_cells);
    s->v = (double *)malloc(sizeof(double) * n_cells);
    s->diff = (double *)malloc(sizeof(double) * n_cells);
    s->fibre = (double *)malloc(sizeof(double) * 3 * n_cells);
    for (int64_t c = 0; c < n_cells; ++c) {
        const orc_cellparams *p = &s->sets[s->pset[c]];
        orc_model_init(p, s->state + ORC_MAXVAR * c);
        double f[3] = {1.0, 0.0, 0.0};
        if (fibre) { f[0] = fibre[3 * c]; f[1] = fibre[3 * c + 1]; f[2] = fibre[3 * c + 2]; }
        memcpy(s->fibre + 3 * c, f, sizeof(f));
        orc_conductivity(f, p->D_l, p->D_t, s->D + 9 * c);
        s->act[c] = INFINITY;
    }
    *err = 0;
    return s;
}

orc_sim *orc_sim_create(int64_t n_nodes, const double *xyz, int64_t n_cells,
                        const int32_t *tet, const double *fibre,
                        const uint8_t *param_set, const uint8_t *stim_mask,
                        int n_sets, const orc_cellparams *sets,
                        int n_stim, const orc_stim *stim,
                        double dt, double threshold, int *err) {
    return orc_sim_create2(n_nodes, xyz, n_cells, tet, 0, NULL, fibre, param_set, stim_mask, n_sets, sets, n_stim,
                           stim, dt, threshold, err);
}

/* The diffusion term of every cell: fv3d.c on the tetrahedra, fv2d.c on the shell. */
static void sim_diffusion(const orc_sim *s, const double *D, const double *v, double *out) {
    if (s->m) orc_diffusion(s->m, D, v, out);
    if (s->shell) orc_shell_diffusion(s->shell, D + 9 * s->n_tets, v + s->n_tets, out + s->n_tets);
}

/* Centroids of all cells (tetrahedra, then shell triangles). */
static void sim_centroids(const orc_sim *s, double *cen) {
    if (s->m) orc_mesh_cell_info(s->m, cen, NULL, NULL);
    if (s->shell) orc_shell_cell_info(s->shell, cen + 3 * s->n_tets, NULL, NULL);
}

void orc_sim_destroy(orc_sim *s) {
    if (!s) return;
    orc_mesh_destroy(s->m);
    orc_shell_destroy(s->shell);
    free(s->xyz);
    orc_graph_free(s->g);
    free(s->i_extra); free(s->s_extra); free(s->vg_old); free(s->v_new);
    free(s->pset); free(s->smask); free(s->state); free(s->D); free(s->act);
    free(s->v); free(s->diff); free(s->fibre);
    free(s->ve); free(s->Die); free(s->u); free(s->rhs); free(s->hist);
    free(s);
}

void orc_sim_run(orc_sim *s, int64_t n_steps) {
    for (int64_t it = 0; it < n_steps; ++it) {
        const int64_t n = s->step;
        const double t = (double)n * s->dt;
        double amp[8];
        for (int k = 0; k < s->n_stim; ++k)
            amp[k] = orc_stim_active(&s->stim[k], s->dt, n) ? s->stim[k].amplitude : 0.0;
        for (int64_t c = 0; c < s->n_cells; ++c) s->v[c] = s->state[ORC_MAXVAR * c];
        if (s->ve) {
            /* bidomain: intracellular flux of V + v_e (first line of Eq. 6) */
            for (int64_t c = 0; c < s->n_cells; ++c) s->u[c] = s->v[c] + s->ve[c];
            sim_diffusion(s, s->D, s->u, s->diff);
        } else {
            sim_diffusion(s, s->D, s->v, s->diff);
        }
        if (s->g) {
            memset(s->i_extra, 0, sizeof(double) * s->n_cells);
            memset(s->s_extra, 0, sizeof(double) * s->n_cells);
            orc_graph_cell_terms(s->g, s->v, t, s->i_extra, s->s_extra);
        }
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < s->n_cells; ++c) {
            double *st = s->state + ORC_MAXVAR * c;
            double is = 0.0, ix = 0.0;
            for (int k = 0; k < s->n_stim; ++k)
                if (s->smask[c] & (1u << k)) is += amp[k];
            if (s->g) {
                is += s->s_extra[c];
                ix = s->i_extra[c];
            }
            const double vn = st[0];
            orc_ab2 ab = {s->hist ? s->hist + (size_t)ORC_NHIST * c : NULL, n > s->ab2_from};
            orc_ab2 *abp = s->integrator ? &ab : NULL;
            const double iion = orc_model_step(st, s->dt, is, &s->sets[s->pset[c]], abp);
            const double vnew = vn + s->dt * orc_rate(abp, 0, s->diff[c] - iion - is - ix);
            st[0] = vnew;
            if (isinf(s->act[c]) && vn < s->theta && vnew >= s->theta)
                s->act[c] = t + s->dt * (s->theta - vn) / (vnew - vn);
        }
        if (s->g) {
            const int64_t ng = orc_graph_n(s->g);
            double *gs = orc_graph_state(s->g);
            for (int64_t i = 0; i < ng; ++i) s->vg_old[i] = gs[ORC_MAXVAR * i];
            orc_graph_step(s->g, s->v, t, s->dt, n, s->sets, s->stim, s->n_stim);
            for (int64_t c = 0; c < s->n_cells; ++c) s->v_new[c] = s->state[ORC_MAXVAR * c];
            orc_graph_triggers(s->g, s->v, s->v_new, s->vg_old, t, s->dt);
        }
        if (s->ve) bidomain_solve(s);
        s->step = n + 1;
    }
}

int orc_sim_attach_graph(orc_sim *s, int64_t n, const double *xyz, int64_t n_edges, const int32_t *edges,
                         const double *edge_D, const uint8_t *pset, const uint8_t *smask,
                         int64_t n_junc, const int32_t *jnode, const int32_t *jcell, const uint8_t *jmode,
                         const orc_graph_params *p) {
    orc_graph_params q = *p;
    q.act_threshold = s->theta;
    double *cen = (double *)malloc(sizeof(double) * 3 * s->n_cells);
    sim_centroids(s, cen);
    int err = 0;
    orc_graph *g = orc_graph_build(n, xyz, n_edges, edges, edge_D, pset, smask, s->n_sets, s->sets, s->dt,
                                   n_junc, jnode, jcell, jmode, &q, s->n_cells, cen, s->n_tets, &err);
    free(cen);
    if (!g) return err;
    orc_graph_free(s->g);
    s->g = g;
    free(s->i_extra); free(s->s_extra); free(s->vg_old); free(s->v_new);
    s->i_extra = (double *)calloc(s->n_cells, sizeof(double));
    s->s_extra = (double *)calloc(s->n_cells, sizeof(double));
    s->v_new = (double *)calloc(s->n_cells, sizeof(double));
    s->vg_old = (double *)calloc(n ? n : 1, sizeof(double));
    return 0;
}

void orc_sim_graph_laplacian(const orc_sim *s, const double *W, double *out) { orc_graph_laplacian(s->g, W, out); }

int orc_sim_graph_substeps(const orc_sim *s) { return s->g ? orc_graph_substeps(s->g) : 0; }

void orc_sim_graph_get_var(const orc_sim *s, int var, double *out) {
    const double *gs = orc_graph_state(s->g);
    for (int64_t i = 0; i < orc_graph_n(s->g); ++i) out[i] = gs[ORC_MAXVAR * i + var];
}

void orc_sim_graph_set_var(orc_sim *s, int var, const double *in) {
    double *gs = orc_graph_state(s->g);
    for (int64_t i = 0; i < orc_graph_n(s->g); ++i) gs[ORC_MAXVAR * i + var] = in[i];
}

void orc_sim_graph_get_act(const orc_sim *s, double *out) {
    memcpy(out, orc_graph_act(s->g), sizeof(double) * orc_graph_n(s->g));
}

int64_t orc_sim_step_index(const orc_sim *s) { return s->step; }
void orc_sim_set_step_index(orc_sim *s, int64_t n) {
    s->step = n;
    s->ab2_from = n;   /* the AB2 history restarts */
}

/* Time integration of the non-gating variables (V and the concentrations):
 * 0 forward Euler (Sec. 3.2), 1 second-order Adams-Bashforth (Sec. 4). The
 * conduction graph's nodes stay forward Euler. AB2 starts from the current
 * step with one forward-Euler step. */
int orc_sim_set_integrator(orc_sim *s, int integrator) {
    if (integrator != 0 && integrator != 1) return 30;
    s->integrator = integrator;
    s->ab2_from = s->step;
    if (integrator && !s->hist) s->hist = (double *)calloc((size_t)ORC_NHIST * s->n_cells, sizeof(double));
    return 0;
}

void orc_sim_get_var(const orc_sim *s, int var, double *out) {
    for (int64_t c = 0; c < s->n_cells; ++c) out[c] = s->state[ORC_MAXVAR * c + var];
}

void orc_sim_set_var(orc_sim *s, int var, const double *in) {
    for (int64_t c = 0; c < s->n_cells; ++c) s->state[ORC_MAXVAR * c + var] = in[c];
    s->ab2_from = s->step;   /* the AB2 history restarts */
}

void orc_sim_get_act(const orc_sim *s, double *out) {
    memcpy(out, s->act, sizeof(double) * s->n_cells);
}

void orc_sim_diffusion(const orc_sim *s, const double *v, double *out) {
    sim_diffusion(s, s->D, v, out);
}

const orc_mesh *orc_sim_mesh(const orc_sim *s) { return s->m; }

/* ---- bidomain (Eq. 1, Eqs. 5-6) -------------------------------------------
 * With the extracellular potential v_e as a second unknown, a step is
 *   V^{n+1} = V^n + dt (L_i(V^n + v_e^n) - I_ion - I_s)
 * followed by the second line of Eq. 6 for v_e^{n+1}:
 *   L_ie(v_e^{n+1}) = -L_i(V^{n+1}),
 * L_i and L_ie being the diffusion operator of fv3d.c with the intracellular
 * tensor D_i and with D_i + D_e. As in Sec. 3.2 the linear system is solved
 * by restarted GMRES started from v_e^n; this is the textbook method
 * (Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
 * matrix), stopped when the true residual satisfies ||b - A x|| <= tol ||b||.
 * v_e is defined up to a constant (zero-flux boundaries everywhere); it is
 * fixed to zero volume-weighted mean after each solve.
 */

static double dot(const double *a, const double *b, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Restarted GMRES on L(D) x = b; returns the iterations (matrix-vector
 * products inside the Arnoldi cycles) and the final relative residual. */
static int64_t gmres(const orc_mesh *m, const double *D, const double *b, double *x, int64_t n, double tol,
                     int restart, int64_t max_iter, double *rel_res, int *failed) {
    const int k = restart;
    double *Vb = (double *)malloc(sizeof(double) * (size_t)(k + 1) * (size_t)n);
    double *H = (double *)calloc((size_t)(k + 1) * k, sizeof(double));   /* H[i * k + j] */
    double *cs = (double *)malloc(sizeof(double) * k), *sn = (double *)malloc(sizeof(double) * k);
    double *g = (double *)malloc(sizeof(double) * (k + 1)), *y = (double *)malloc(sizeof(double) * k);
    double *w = (double *)malloc(sizeof(double) * n);
    const double bnorm = sqrt(dot(b, b, n));
    int64_t it = 0;
    *failed = 0;
    *rel_res = 0.0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
    } else {
        for (;;) {
            /* true residual r = b - A x, into the first basis vector */
            double *v0 = Vb;
            orc_diffusion(m, D, x, v0);
            for (int64_t i = 0; i < n; ++i) v0[i] = b[i] - v0[i];
            const double beta = sqrt(dot(v0, v0, n));
            *rel_res = beta / bnorm;
            if (beta <= tol * bnorm) break;
            if (it >= max_iter) {
                *failed = 1;
                break;
            }
            for (int64_t i = 0; i < n; ++i) v0[i] /= beta;
            for (int i = 0; i <= k; ++i) g[i] = 0.0;
            g[0] = beta;
            int j = 0;
            while (j < k && it < max_iter) {
                double *vj = Vb + (size_t)j * n, *vn = Vb + (size_t)(j + 1) * n;
                orc_diffusion(m, D, vj, w);
                ++it;
                for (int i = 0; i <= j; ++i) {          /* modified Gram-Schmidt */
                    const double *vi = Vb + (size_t)i * n;
                    const double h = dot(w, vi, n);
                    H[i * k + j] = h;
                    for (int64_t r = 0; r < n; ++r) w[r] -= h * vi[r];
                }
                const double hn = sqrt(dot(w, w, n));
                H[(j + 1) * k + j] = hn;
                for (int64_t r = 0; r < n; ++r) vn[r] = hn > 0.0 ? w[r] / hn : 0.0;
                for (int i = 0; i < j; ++i) {           /* earlier rotations on column j */
                    const double a = H[i * k + j], c = H[(i + 1) * k + j];
                    H[i * k + j] = cs[i] * a + sn[i] * c;
                    H[(i + 1) * k + j] = -sn[i] * a + cs[i] * c;
                }
                const double a = H[j * k + j], c = H[(j + 1) * k + j];
                const double rr = sqrt(a * a + c * c);
                cs[j] = rr > 0.0 ? a / rr : 1.0;
                sn[j] = rr > 0.0 ? c / rr : 0.0;
                H[j * k + j] = rr;
                H[(j + 1) * k + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                ++j;
                if (fabs(g[j]) <= tol * bnorm || hn == 0.0) break;
            }
            /* x += V_j y, H_j y = g (upper triangular) */
            for (int i = j - 1; i >= 0; --i) {
                double sacc = g[i];
                for (int l = i + 1; l < j; ++l) sacc -= H[i * k + l] * y[l];
                y[i] = H[i * k + i] != 0.0 ? sacc / H[i * k + i] : 0.0;
            }
            for (int i = 0; i < j; ++i) {
                const double *vi = Vb + (size_t)i * n;
                for (int64_t r = 0; r < n; ++r) x[r] += y[i] * vi[r];
            }
        }
    }
    free(Vb); free(H); free(cs); free(sn); free(g); free(y); free(w);
    return it;
}

static void bidomain_solve(orc_sim *s) {
    const int64_t n = s->n_cells;
    for (int64_t c = 0; c < n; ++c) s->v[c] = s->state[ORC_MAXVAR * c];
    orc_diffusion(s->m, s->D, s->v, s->rhs);
    for (int64_t c = 0; c < n; ++c) s->rhs[c] = -s->rhs[c];
    int failed = 0;
    s->gm_last_iter = gmres(s->m, s->Die, s->rhs, s->ve, n, s->gm_tol, s->gm_restart, s->gm_max_iter,
                            &s->gm_last_res, &failed);
    s->gm_total_iter += s->gm_last_iter;
    s->gm_failed |= failed;
    /* gauge: zero volume-weighted mean */
    double sv = 0.0, sw = 0.0;
    double *vol = s->u;   /* scratch */
    orc_mesh_cell_info(s->m, NULL, vol, NULL);
    for (int64_t c = 0; c < n; ++c) {
        sv += vol[c] * s->ve[c];
        sw += vol[c];
    }
    for (int64_t c = 0; c < n; ++c) s->ve[c] -= sv / sw;
}

/* Switch the simulation to the bidomain model: the parameter sets' (D_l,
 * D_t) become the intracellular diffusivities, De_l[k], De_t[k] are the
 * extracellular ones of set k (mm^2/ms, both tensors in the cell's fibre
 * frame, Eqs. 2-3). v_e is solved at once from the current V (from x = 0).
 * tol, restart, max_iter: the GMRES stopping rule, Krylov dimension and
 * iteration cap per solve. */
int orc_sim_set_bidomain(orc_sim *s, const double *De_l, const double *De_t, double tol, int restart,
                         int64_t max_iter) {
    if (!(tol > 0.0) || restart < 1 || max_iter < 1) return 20;
    if (s->shell || !s->m) return 21;   /* the Purkinje shell is a monodomain medium (Table 2) */
    const int64_t n = s->n_cells;
    free(s->ve); free(s->Die); free(s->u); free(s->rhs);
    s->ve = (double *)calloc(n, sizeof(double));
    s->Die = (double *)malloc(sizeof(double) * 9 * n);
    s->u = (double *)malloc(sizeof(double) * n);
    s->rhs = (double *)malloc(sizeof(double) * n);
    for (int64_t c = 0; c < n; ++c) {
        const orc_cellparams *p = &s->sets[s->pset[c]];
        const int k = s->pset[c];
        orc_conductivity(s->fibre + 3 * c, p->D_l + De_l[k], p->D_t + De_t[k], s->Die + 9 * c);
    }
    s->gm_tol = tol;
    s->gm_restart = restart;
    s->gm_max_iter = max_iter;
    s->gm_total_iter = 0;
    s->gm_failed = 0;
    bidomain_solve(s);
    return 0;
}

void orc_sim_get_ve(const orc_sim *s, double *out) {
    if (s->ve) memcpy(out, s->ve, sizeof(double) * s->n_cells);
    else memset(out, 0, sizeof(double) * s->n_cells);
}

void orc_sim_set_ve(orc_sim *s, const double *in) {
    if (s->ve) memcpy(s->ve, in, sizeof(double) * s->n_cells);
}

/* stats[0] iterations of the last solve, [1] all iterations, [2] the last
 * relative residual, [3] 1 if a solve hit its iteration cap. */
void orc_sim_bidomain_stats(const orc_sim *s, double *stats) {
    stats[0] = (double)s->gm_last_iter;
    stats[1] = (double)s->gm_total_iter;
    stats[2] = s->gm_last_res;
    stats[3] = (double)s->gm_failed;
}

/* The elliptic operator alone: out = L_ie(x) (a check of the solve). */
void orc_sim_bidomain_operator(const orc_sim *s, const double *x, double *out) {
    orc_diffusion(s->m, s->Die, x, out);
}
