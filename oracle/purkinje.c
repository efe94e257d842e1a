/*
 * Oracle (test infrastructure only): the 1D conduction graph and its
 * junctions with the myocardium.
 *
 * Graph (Sec. 3.2, vertex-based FV for 1D media, branches allowed at a node):
 * node i has the control length V_i = (1/2) sum_j L_ij over its edges, and
 * the flux along edge ij is D_ij (V_j - V_i) / L_ij, so
 *     dV_i/dt = (2 / sum_j L_ij) sum_j D_ij (V_j - V_i) / L_ij - I_ion - I_s.
 * Every node carries a cell model (its parameter set's model) advanced by
 * RL / FE at (V^n, s^n). The diffusion is subcycled: with the reaction
 * (ionic, stimulus and junction currents) frozen at step n, k substeps of
 * h = dt / k advance V, where k = max(1, ceil(dt * rho / 1.8)) and
 * rho = max_i 2 sum_j c_ij bounds the graph operator's spectrum
 * (c_ij = 2 D_ij / (L_ij sum_k L_ik)).
 *
 * Junctions (Sec. 3.3) pair a graph node p with a myocardial cell m:
 *  - resistive: the current g_graph (V_p - V_m) leaves node p and
 *    g_cell (V_m - V_p) leaves cell m, both evaluated at step n;
 *  - triggered: each upward crossing of the threshold by V_p at time t_p
 *    (interpolated within the step) makes the stimulus `amplitude` act on
 *    every cell of cell m's medium (myocardium or Purkinje shell) whose
 *    centroid lies within `radius` of cell m's centroid
 *    while t_p + delay_ortho <= t < t_p + delay_ortho + duration; with
 *    two_way, each upward crossing by V_m at t_m likewise stimulates node p
 *    over [t_m + delay_anti, t_m + delay_anti + duration).
 *    Crossings found in step n act from step n + 1 on.
 * Communication nodes between two cells (Sec. 3.3: the 2D Purkinje shell and
 * the 3D myocardium) work like the triggered junction with a source cell s
 * (given in place of the graph node) instead of node p: each upward crossing
 * by V_s stimulates the cells within `radius` of cell m after delay_ortho;
 * with two_way, crossings by V_m stimulate cell s after delay_anti.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

struct orc_graph {
    int64_t n;
    double *state;      /* [n][ORC_MAXVAR]; variable 0 is V */
    uint8_t *pset, *smask;
    int64_t *ptr;       /* CSR of neighbours */
    int32_t *nbr;
    double *coef;       /* c_ij */
    int substeps;
    double *act;
    int64_t n_junc;
    int32_t *jnode, *jcell;
    uint8_t *jmode;
    double *t_graph, *t_cell;   /* last upward crossing times, -inf if none */
    int64_t *tgt_ptr;           /* triggered junction j -> target cells */
    int32_t *tgt;
    orc_graph_params p;
};

void orc_graph_free(orc_graph *g) {
    if (!g) return;
    free(g->state); free(g->pset); free(g->smask); free(g->ptr); free(g->nbr); free(g->coef);
    free(g->act); free(g->jnode); free(g->jcell); free(g->jmode); free(g->t_graph); free(g->t_cell);
    free(g->tgt_ptr); free(g->tgt);
    free(g);
}

orc_graph *orc_graph_build(int64_t n, const double *xyz, int64_t n_edges, const int32_t *edges,
                           const double *edge_D, const uint8_t *pset, const uint8_t *smask,
                           int n_sets, const orc_cellparams *sets, double dt,
                           int64_t n_junc, const int32_t *jnode, const int32_t *jcell,
                           const uint8_t *jmode, const orc_graph_params *p,
                           int64_t n_cells, const double *cell_centroid, int64_t n_tets, int *err) {
    *err = 0;
    for (int64_t e = 0; e < n_edges; ++e)
        if (edges[2 * e] < 0 || edges[2 * e] >= n || edges[2 * e + 1] < 0 || edges[2 * e + 1] >= n ||
            edges[2 * e] == edges[2 * e + 1]) { *err = 20; return NULL; }
    for (int64_t i = 0; i < n; ++i)
        if (pset && pset[i] >= n_sets) { *err = 21; return NULL; }
    for (int64_t j = 0; j < n_junc; ++j) {
        const int cellsrc = jmode && jmode[j] == ORC_JUNC_CELL;
        if (jnode[j] < 0 || jnode[j] >= (cellsrc ? n_cells : n) || jcell[j] < 0 || jcell[j] >= n_cells ||
            (jmode && jmode[j] > ORC_JUNC_CELL)) { *err = 22; return NULL; }
    }
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    g->n = n;
    g->p = *p;
    g->state = (double *)calloc(ORC_MAXVAR * (size_t)n, sizeof(double));
    g->pset = (uint8_t *)calloc(n, 1);
    g->smask = (uint8_t *)calloc(n, 1);
    if (pset) memcpy(g->pset, pset, n);
    if (smask) memcpy(g->smask, smask, n);
    g->act = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) {
        orc_model_init(&sets[g->pset[i]], g->state + ORC_MAXVAR * i);
        g->act[i] = INFINITY;
    }
    /* adjacency and the control length of each node */
    g->ptr = (int64_t *)calloc(n + 1, sizeof(int64_t));
    for (int64_t e = 0; e < n_edges; ++e) { g->ptr[edges[2 * e] + 1]++; g->ptr[edges[2 * e + 1] + 1]++; }
    for (int64_t i = 0; i < n; ++i) g->ptr[i + 1] += g->ptr[i];
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * 2 * (n_edges ? n_edges : 1));
    double *len = (double *)malloc(sizeof(double) * 2 * (n_edges ? n_edges : 1));
    double *dif = (double *)malloc(sizeof(double) * 2 * (n_edges ? n_edges : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    memcpy(fill, g->ptr, sizeof(int64_t) * n);
    for (int64_t e = 0; e < n_edges; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1], dz = xyz[3 * a + 2] - xyz[3 * b + 2];
        double L = sqrt(dx * dx + dy * dy + dz * dz);
        double D = edge_D ? edge_D[e] : p->D;
        g->nbr[fill[a]] = b; len[fill[a]] = L; dif[fill[a]] = D; fill[a]++;
        g->nbr[fill[b]] = a; len[fill[b]] = L; dif[fill[b]] = D; fill[b]++;
    }
    free(fill);
    g->coef = (double *)malloc(sizeof(double) * 2 * (n_edges ? n_edges : 1));
    double rho = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double sumL = 0.0;
        for (int64_t k = g->ptr[i]; k < g->ptr[i + 1]; ++k) sumL += len[k];
        double row = 0.0;
        for (int64_t k = g->ptr[i]; k < g->ptr[i + 1]; ++k) {
            g->coef[k] = 2.0 * dif[k] / (len[k] * sumL);
            row += g->coef[k];
        }
        if (2.0 * row > rho) rho = 2.0 * row;
    }
    free(len);
    free(dif);
    g->substeps = (int)ceil(dt * rho / 1.8);
    if (g->substeps < 1) g->substeps = 1;
    /* junctions and the target cells of triggered ones */
    g->n_junc = n_junc;
    g->jnode = (int32_t *)malloc(sizeof(int32_t) * (n_junc ? n_junc : 1));
    g->jcell = (int32_t *)malloc(sizeof(int32_t) * (n_junc ? n_junc : 1));
    g->jmode = (uint8_t *)calloc(n_junc ? n_junc : 1, 1);
    g->t_graph = (double *)malloc(sizeof(double) * (n_junc ? n_junc : 1));
    g->t_cell = (double *)malloc(sizeof(double) * (n_junc ? n_junc : 1));
    g->tgt_ptr = (int64_t *)calloc(n_junc + 1, sizeof(int64_t));
    if (n_junc) {
        memcpy(g->jnode, jnode, sizeof(int32_t) * n_junc);
        memcpy(g->jcell, jcell, sizeof(int32_t) * n_junc);
        if (jmode) memcpy(g->jmode, jmode, n_junc);
    }
    int64_t cap = 16, cnt = 0;
    g->tgt = (int32_t *)malloc(sizeof(int32_t) * cap);
    for (int64_t j = 0; j < n_junc; ++j) {
        g->t_graph[j] = -INFINITY;
        g->t_cell[j] = -INFINITY;
        if (g->jmode[j] == ORC_JUNC_TRIGGERED || g->jmode[j] == ORC_JUNC_CELL) {
            const double *x0 = cell_centroid + 3 * (int64_t)jcell[j];
            const int shell = jcell[j] >= n_tets;   /* targets: cells of the target cell's medium */
            for (int64_t c = 0; c < n_cells; ++c) {
                if ((c >= n_tets) != shell) continue;
                const double *x = cell_centroid + 3 * c;
                double dx = x[0] - x0[0], dy = x[1] - x0[1], dz = x[2] - x0[2];
                if (c == jcell[j] || sqrt(dx * dx + dy * dy + dz * dz) <= p->radius) {
                    if (cnt == cap) { cap *= 2; g->tgt = (int32_t *)realloc(g->tgt, sizeof(int32_t) * cap); }
                    g->tgt[cnt++] = (int32_t)c;
                }
            }
        }
        g->tgt_ptr[j + 1] = cnt;
    }
    return g;
}

int orc_graph_substeps(const orc_graph *g) { return g->substeps; }
int64_t orc_graph_n(const orc_graph *g) { return g->n; }
double *orc_graph_state(orc_graph *g) { return g->state; }
double *orc_graph_act(orc_graph *g) { return g->act; }

static int window_on(double t_trig, double delay, double dur, double t) {
    return isfinite(t_trig) && t >= t_trig + delay && t < t_trig + delay + dur;
}

/* Extra current (resistive) and stimulus (triggered) on 3D cells at step n. */
void orc_graph_cell_terms(const orc_graph *g, const double *V, double t, double *i_extra, double *s_extra) {
    for (int64_t j = 0; j < g->n_junc; ++j) {
        const int32_t p = g->jnode[j], m = g->jcell[j];
        if (g->jmode[j] == ORC_JUNC_RESISTIVE) {
            i_extra[m] += g->p.g_cell * (V[m] - g->state[ORC_MAXVAR * (int64_t)p]);
            continue;
        }
        if (window_on(g->t_graph[j], g->p.delay_ortho, g->p.duration, t))
            for (int64_t k = g->tgt_ptr[j]; k < g->tgt_ptr[j + 1]; ++k) s_extra[g->tgt[k]] += g->p.amplitude;
        /* the source cell of a cell-to-cell node, excited back (two-way) */
        if (g->jmode[j] == ORC_JUNC_CELL && g->p.two_way && window_on(g->t_cell[j], g->p.delay_anti, g->p.duration, t))
            s_extra[p] += g->p.amplitude;
    }
}

/* Advance the graph one step from (V^n, s^n) given the 3D V^n. */
void orc_graph_step(orc_graph *g, const double *V3, double t, double dt, int64_t n_step,
                    const orc_cellparams *sets, const orc_stim *stim, int n_stim) {
    const int64_t n = g->n;
    double *itot = (double *)calloc(n ? n : 1, sizeof(double));
    double *sx = (double *)calloc(n ? n : 1, sizeof(double));
    double *W = (double *)malloc(sizeof(double) * (n ? n : 1));
    double *W2 = (double *)malloc(sizeof(double) * (n ? n : 1));
    /* junction terms on the graph side, at step n */
    for (int64_t j = 0; j < g->n_junc; ++j) {
        const int32_t p = g->jnode[j], m = g->jcell[j];
        if (g->jmode[j] == ORC_JUNC_RESISTIVE)
            itot[p] += g->p.g_graph * (g->state[ORC_MAXVAR * (int64_t)p] - V3[m]);
        else if (g->jmode[j] == ORC_JUNC_TRIGGERED && g->p.two_way &&
                 window_on(g->t_cell[j], g->p.delay_anti, g->p.duration, t))
            sx[p] += g->p.amplitude;
    }
    /* reaction at (V^n, s^n), frozen over the substeps */
    for (int64_t i = 0; i < n; ++i) {
        double *st = g->state + ORC_MAXVAR * i;
        double is = sx[i];
        for (int k = 0; k < n_stim; ++k)
            if ((g->smask[i] >> k) & 1u)
                if (orc_stim_active(&stim[k], dt, n_step)) is += stim[k].amplitude;
        W[i] = st[0];
        const double iion = orc_model_step(st, dt, is, &sets[g->pset[i]], NULL);
        itot[i] += iion + is;
    }
    const double h = dt / g->substeps;
    for (int s = 0; s < g->substeps; ++s) {
        for (int64_t i = 0; i < n; ++i) {
            double lap = 0.0;
            for (int64_t k = g->ptr[i]; k < g->ptr[i + 1]; ++k) lap += g->coef[k] * (W[g->nbr[k]] - W[i]);
            W2[i] = W[i] + h * (lap - itot[i]);
        }
        double *tmp = W; W = W2; W2 = tmp;
    }
    /* V^{n+1}, activation and triggers of the graph side */
    for (int64_t i = 0; i < n; ++i) {
        double *st = g->state + ORC_MAXVAR * i;
        const double v0 = st[0], v1 = W[i];
        st[0] = v1;
        if (isinf(g->act[i]) && v0 < g->p.act_threshold && v1 >= g->p.act_threshold)
            g->act[i] = t + dt * (g->p.act_threshold - v0) / (v1 - v0);
    }
    free(itot); free(sx); free(W); free(W2);
}

/* Record upward threshold crossings of triggered junctions (both sides)
 * between V^n and V^{n+1}. */
void orc_graph_triggers(orc_graph *g, const double *V3_old, const double *V3_new, const double *Vg_old,
                        double t, double dt) {
    const double th = g->p.threshold;
    for (int64_t j = 0; j < g->n_junc; ++j) {
        if (g->jmode[j] == ORC_JUNC_RESISTIVE) continue;
        const int cellsrc = g->jmode[j] == ORC_JUNC_CELL;   /* the source is a cell, not a graph node */
        const double a = cellsrc ? V3_old[g->jnode[j]] : Vg_old[g->jnode[j]];
        const double b = cellsrc ? V3_new[g->jnode[j]] : g->state[ORC_MAXVAR * (int64_t)g->jnode[j]];
        if (a < th && b >= th) g->t_graph[j] = t + dt * (th - a) / (b - a);
        const double c = V3_old[g->jcell[j]], d = V3_new[g->jcell[j]];
        if (g->p.two_way && c < th && d >= th) g->t_cell[j] = t + dt * (th - c) / (d - c);
    }
}

/* The graph diffusion operator alone: out_i = sum_j c_ij (W_j - W_i). */
void orc_graph_laplacian(const orc_graph *g, const double *W, double *out) {
    for (int64_t i = 0; i < g->n; ++i) {
        double lap = 0.0;
        for (int64_t k = g->ptr[i]; k < g->ptr[i + 1]; ++k) lap += g->coef[k] * (W[g->nbr[k]] - W[i]);
        out[i] = lap;
    }
}
