/*
 * Oracle (test infrastructure only): the 2D Purkinje shell (Sec. 2, Sec.
 * 3.2), a surface of triangles in 3D space discretised by the same
 * cell-centred finite-volume scheme as the myocardium, with edges as faces:
 *
 *   S1  node value   v_n = sum_k v_k / d_k  /  sum_k 1 / d_k      (triangles k around n,
 *                    d_k = |x_n - x_k|, the distance to the triangle centroid)
 *   S2  edge value   v_f = mean of the two end-node values
 *       cell gradient  grad v_c = (1/A_c) sum_j v_fj L_fj n_fj   (Gauss-Green in the
 *                    triangle's plane, n_fj the outward in-plane edge normal)
 *   S3  edge gradient  gbar_f = a_c1 grad v_c1 + a_c2 grad v_c2,
 *       corrected      grad v_f = gbar_f + [(v_c1 - v_c2)/d - gbar_f.e] e       (Eq. 8)
 *       flux           L_f (D_f grad v_f) . n_f, summed over the cell's edges, / A_c
 *
 * Readings taken where the paper is silent (beyond those of fv3d.c):
 *   - on a curved surface the two triangles of an edge lie in different
 *     planes; the edge normal used for the flux is the normalised mean of
 *     the first triangle's outward normal and the negated outward normal of
 *     the second, so the edge flux leaving one cell enters the other exactly;
 *     a_c1 and x_f use the edge midpoint;
 *   - the conductivity tensor is the cell's (D_t I + (D_l - D_t) f f^T), the
 *     Purkinje shell taking D_l = D_t (isotropic, Table 2);
 *   - boundary edges carry zero flux.
 * The result returned is the diffusion term of dV/dt.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

struct orc_shell {
    int64_t n_nodes, n_cells;
    const double *xyz;  /* borrowed: [3 n_nodes] */
    int32_t *tri;       /* [3 n_cells] */
    double *xc;         /* [3 n_cells] centroid */
    double *area;       /* [n_cells] */
    double *un;         /* [3 n_cells] unit normal of the triangle's plane */
    int32_t *nb;        /* [3 n_cells] triangle across the edge opposite vertex i, -1 on the boundary */
    double *len;        /* [3 n_cells] edge length */
    double *en;         /* [9 n_cells] outward in-plane unit normal of edge i */
    double *xf;         /* [9 n_cells] edge midpoint */
    int64_t *n2c_ptr;   /* [n_nodes + 1] triangles around each node */
    int32_t *n2c;
};

static double dist3(const double *a, const double *b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

void orc_shell_destroy(orc_shell *s) {
    if (!s) return;
    free(s->tri); free(s->xc); free(s->area); free(s->un); free(s->nb); free(s->len); free(s->en);
    free(s->xf); free(s->n2c_ptr); free(s->n2c);
    free(s);
}

/* err: 1 node index out of range, 2 degenerate triangle, 3 edge shared by more than two triangles */
orc_shell *orc_shell_create(int64_t n_nodes, const double *xyz, int64_t n_cells, const int32_t *tri, int *err) {
    *err = 0;
    for (int64_t i = 0; i < 3 * n_cells; ++i)
        if (tri[i] < 0 || tri[i] >= n_nodes) { *err = 1; return NULL; }
    orc_shell *s = (orc_shell *)calloc(1, sizeof(orc_shell));
    s->n_nodes = n_nodes;
    s->n_cells = n_cells;
    s->xyz = xyz;
    s->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * n_cells);
    memcpy(s->tri, tri, sizeof(int32_t) * 3 * n_cells);
    s->xc = (double *)malloc(sizeof(double) * 3 * n_cells);
    s->area = (double *)malloc(sizeof(double) * n_cells);
    s->un = (double *)malloc(sizeof(double) * 3 * n_cells);
    s->nb = (int32_t *)malloc(sizeof(int32_t) * 3 * n_cells);
    s->len = (double *)malloc(sizeof(double) * 3 * n_cells);
    s->en = (double *)malloc(sizeof(double) * 9 * n_cells);
    s->xf = (double *)malloc(sizeof(double) * 9 * n_cells);
    for (int64_t c = 0; c < n_cells; ++c) {
        const double *p[3];
        for (int k = 0; k < 3; ++k) p[k] = xyz + 3 * (int64_t)tri[3 * c + k];
        double u[3], v[3], w[3];
        for (int k = 0; k < 3; ++k) {
            s->xc[3 * c + k] = (p[0][k] + p[1][k] + p[2][k]) / 3.0;
            u[k] = p[1][k] - p[0][k];
            v[k] = p[2][k] - p[0][k];
        }
        w[0] = u[1] * v[2] - u[2] * v[1];
        w[1] = u[2] * v[0] - u[0] * v[2];
        w[2] = u[0] * v[1] - u[1] * v[0];
        double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        double lmax = fmax(dist3(p[0], p[1]), fmax(dist3(p[1], p[2]), dist3(p[0], p[2])));
        if (!(nw > 1e-12 * lmax * lmax)) { *err = 2; orc_shell_destroy(s); return NULL; }
        s->area[c] = 0.5 * nw;
        for (int k = 0; k < 3; ++k) s->un[3 * c + k] = w[k] / nw;
        /* edge i joins the two vertices other than i */
        for (int i = 0; i < 3; ++i) {
            const double *a = p[(i + 1) % 3], *b = p[(i + 2) % 3];
            double t[3], m[3];
            for (int k = 0; k < 3; ++k) {
                t[k] = b[k] - a[k];
                m[k] = 0.5 * (a[k] + b[k]);
            }
            double L = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
            /* in-plane normal: t x un, turned away from vertex i */
            const double *un = s->un + 3 * c;
            double n[3] = {t[1] * un[2] - t[2] * un[1], t[2] * un[0] - t[0] * un[2], t[0] * un[1] - t[1] * un[0]};
            double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            double away = 0.0;
            for (int k = 0; k < 3; ++k) away += n[k] * (m[k] - p[i][k]);
            for (int k = 0; k < 3; ++k) {
                s->en[9 * c + 3 * i + k] = (away < 0 ? -n[k] : n[k]) / nn;
                s->xf[9 * c + 3 * i + k] = m[k];
            }
            s->len[3 * c + i] = L;
            s->nb[3 * c + i] = -1;
        }
    }
    /* edge matching: brute force through the node -> triangle incidence */
    s->n2c_ptr = (int64_t *)calloc(n_nodes + 1, sizeof(int64_t));
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < 3; ++k) s->n2c_ptr[tri[3 * c + k] + 1]++;
    for (int64_t n = 0; n < n_nodes; ++n) s->n2c_ptr[n + 1] += s->n2c_ptr[n];
    s->n2c = (int32_t *)malloc(sizeof(int32_t) * 3 * (n_cells ? n_cells : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n_nodes + 1));
    memcpy(fill, s->n2c_ptr, sizeof(int64_t) * (n_nodes + 1));
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < 3; ++k) s->n2c[fill[tri[3 * c + k]]++] = (int32_t)c;
    free(fill);
    for (int64_t c = 0; c < n_cells; ++c)
        for (int i = 0; i < 3; ++i) {
            int32_t a = tri[3 * c + (i + 1) % 3], b = tri[3 * c + (i + 2) % 3];
            int found = 0;
            for (int64_t j = s->n2c_ptr[a]; j < s->n2c_ptr[a + 1]; ++j) {
                int32_t o = s->n2c[j];
                if (o == c) continue;
                int hasb = 0;
                for (int k = 0; k < 3; ++k) hasb |= tri[3 * (int64_t)o + k] == b;
                if (hasb) {
                    s->nb[3 * c + i] = o;
                    ++found;
                }
            }
            if (found > 1) { *err = 3; orc_shell_destroy(s); return NULL; }
        }
    return s;
}

/* S1 over the shell's nodes (nodes of no triangle get 0). */
void orc_shell_node_values(const orc_shell *s, const double *v, double *vn) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < s->n_nodes; ++n) {
        double num = 0.0, den = 0.0;
        for (int64_t k = s->n2c_ptr[n]; k < s->n2c_ptr[n + 1]; ++k) {
            int32_t c = s->n2c[k];
            double w = 1.0 / dist3(s->xyz + 3 * n, s->xc + 3 * (int64_t)c);
            num += w * v[c];
            den += w;
        }
        vn[n] = den > 0.0 ? num / den : 0.0;
    }
}

/* S2: Gauss-Green gradient of each triangle from its edge values. */
void orc_shell_gradients(const orc_shell *s, const double *vn, double *grad) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < s->n_cells; ++c) {
        double g[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            double vf = 0.5 * (vn[s->tri[3 * c + (i + 1) % 3]] + vn[s->tri[3 * c + (i + 2) % 3]]);
            for (int k = 0; k < 3; ++k) g[k] += vf * s->len[3 * c + i] * s->en[9 * c + 3 * i + k];
        }
        for (int k = 0; k < 3; ++k) grad[3 * c + k] = g[k] / s->area[c];
    }
}

/* S3 and the flux sum: the diffusion term of every triangle. D: [9 n_cells]. */
void orc_shell_diffusion(const orc_shell *s, const double *D, const double *v, double *out) {
    double *vn = (double *)malloc(sizeof(double) * (s->n_nodes ? s->n_nodes : 1));
    double *grad = (double *)malloc(sizeof(double) * 3 * (s->n_cells ? s->n_cells : 1));
    orc_shell_node_values(s, v, vn);
    orc_shell_gradients(s, vn, grad);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < s->n_cells; ++c) {
        double sum = 0.0;
        for (int i = 0; i < 3; ++i) {
            int32_t c2 = s->nb[3 * c + i];
            if (c2 < 0) continue;
            /* the neighbour's edge with this cell, for the shared normal */
            int i2 = 0;
            for (int k = 0; k < 3; ++k)
                if (s->nb[3 * (int64_t)c2 + k] == c) i2 = k;
            double n[3], nn = 0.0;
            for (int k = 0; k < 3; ++k) {
                n[k] = s->en[9 * c + 3 * i + k] - s->en[9 * (int64_t)c2 + 3 * i2 + k];
                nn += n[k] * n[k];
            }
            nn = sqrt(nn);
            for (int k = 0; k < 3; ++k) n[k] /= nn;
            const double *x1 = s->xc + 3 * c, *x2 = s->xc + 3 * (int64_t)c2, *xf = s->xf + 9 * c + 3 * i;
            double r1 = dist3(x1, xf), r2 = dist3(x2, xf);
            double a1 = r2 / (r1 + r2), a2 = 1.0 - a1;
            double d = dist3(x1, x2);
            double e[3], gbar[3], gf[3];
            for (int k = 0; k < 3; ++k) {
                e[k] = (x1[k] - x2[k]) / d;
                gbar[k] = a1 * grad[3 * c + k] + a2 * grad[3 * (int64_t)c2 + k];
            }
            double ge = gbar[0] * e[0] + gbar[1] * e[1] + gbar[2] * e[2];
            double corr = (v[c] - v[c2]) / d - ge;
            for (int k = 0; k < 3; ++k) gf[k] = gbar[k] + corr * e[k];
            double flux = 0.0;
            for (int r = 0; r < 3; ++r) {
                double Dg = 0.0;
                for (int k = 0; k < 3; ++k) Dg += (a1 * D[9 * c + 3 * r + k] + a2 * D[9 * (int64_t)c2 + 3 * r + k]) * gf[k];
                flux += Dg * n[r];
            }
            sum += s->len[3 * c + i] * flux;
        }
        out[c] = sum / s->area[c];
    }
    free(vn);
    free(grad);
}

void orc_shell_cell_info(const orc_shell *s, double *centroid, double *area, int32_t *neighbour) {
    if (centroid) memcpy(centroid, s->xc, sizeof(double) * 3 * s->n_cells);
    if (area) memcpy(area, s->area, sizeof(double) * s->n_cells);
    if (neighbour) memcpy(neighbour, s->nb, sizeof(int32_t) * 3 * s->n_cells);
}
