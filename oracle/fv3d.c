/*
 * Oracle (test infrastructure only): geometry of the cell-centred
 * tetrahedral finite-volume mesh and the diffusion operator of the
 * monodomain equation, written stage by stage as Sec. 3.2 states it.
 *
 *   S1  node value   v_n = sum_k v_k / d_k  /  sum_k 1 / d_k      (cells k around n,
 *                    d_k = |x_n - x_k|, the distance to the cell centre)
 *   S2  face value   v_f = mean of the three vertex values of the face
 *       cell gradient  grad v_c = (1/V_c) sum_j v_fj S_fj n_fj  (Gauss-Green)
 *   S3  face gradient  gbar_f = a_c1 grad v_c1 + a_c2 grad v_c2,  a_c1 + a_c2 = 1
 *       corrected     grad v_f = gbar_f + [(v_c1 - v_c2)/d - gbar_f.e] e    (Eq. 8)
 *       flux           A_f (D_f grad v_f) . n_f, summed over the cell's faces (Eq. 7)
 *
 * Readings taken where the paper is silent:
 *   - e points from the neighbour c2 to the cell c1 itself, d = |x_c1 - x_c2|;
 *   - the linear interpolation weight of c1 at the face is
 *     a_c1 = |x_c2 - x_f| / (|x_c1 - x_f| + |x_c2 - x_f|), x_f the face centroid;
 *   - the face tensor is D_f = a_c1 D_c1 + a_c2 D_c2;
 *   - boundary faces carry zero flux.
 * The result returned is the diffusion term of dV/dt, (1/V_c) sum_j flux_j.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

struct orc_mesh {
    int64_t n_nodes, n_cells;
    double *xyz;       /* [3 n_nodes] */
    int32_t *tet;      /* [4 n_cells] */
    double *xc;        /* [3 n_cells] cell centroid */
    double *vol;       /* [n_cells]   cell volume */
    int32_t *nb;       /* [4 n_cells] cell across the face opposite vertex i, -1 on the boundary */
    double *area;      /* [4 n_cells] face area */
    double *nrm;       /* [12 n_cells] outward unit normal of face i */
    double *xf;        /* [12 n_cells] face centroid */
    int64_t *n2c_ptr;  /* [n_nodes + 1] cells around each node */
    int32_t *n2c;
    int64_t n_boundary;
};

typedef struct { int32_t a, b, c, cell, local; } face_key;

static int cmp_face(const void *p, const void *q) {
    const face_key *x = (const face_key *)p, *y = (const face_key *)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return x->local - y->local;
}

static void sort3(int32_t *v) {
    int32_t t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

void orc_mesh_destroy(orc_mesh *m) {
    if (!m) return;
    free(m->xyz); free(m->tet); free(m->xc); free(m->vol); free(m->nb);
    free(m->area); free(m->nrm); free(m->xf); free(m->n2c_ptr); free(m->n2c);
    free(m);
}

orc_mesh *orc_mesh_create(int64_t n_nodes, const double *xyz, int64_t n_cells,
                          const int32_t *tet, int *err) {
    *err = 0;
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    m->n_nodes = n_nodes;
    m->n_cells = n_cells;
    m->xyz = (double *)malloc(sizeof(double) * 3 * n_nodes);
    memcpy(m->xyz, xyz, sizeof(double) * 3 * n_nodes);
    m->tet = (int32_t *)malloc(sizeof(int32_t) * 4 * n_cells);
    memcpy(m->tet, tet, sizeof(int32_t) * 4 * n_cells);
    m->xc = (double *)malloc(sizeof(double) * 3 * n_cells);
    m->vol = (double *)malloc(sizeof(double) * n_cells);
    m->nb = (int32_t *)malloc(sizeof(int32_t) * 4 * n_cells);
    m->area = (double *)malloc(sizeof(double) * 4 * n_cells);
    m->nrm = (double *)malloc(sizeof(double) * 12 * n_cells);
    m->xf = (double *)malloc(sizeof(double) * 12 * n_cells);

    for (int64_t c = 0; c < n_cells; ++c) {
        for (int i = 0; i < 4; ++i) {
            int32_t v = tet[4 * c + i];
            if (v < 0 || v >= n_nodes) { *err = 1; orc_mesh_destroy(m); return NULL; }
        }
    }

    /* centroid and volume of each tetrahedron */
    for (int64_t c = 0; c < n_cells; ++c) {
        const double *p[4];
        for (int i = 0; i < 4; ++i) p[i] = xyz + 3 * (int64_t)tet[4 * c + i];
        for (int k = 0; k < 3; ++k)
            m->xc[3 * c + k] = 0.25 * (p[0][k] + p[1][k] + p[2][k] + p[3][k]);
        double a[3], b[3], d[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = p[1][k] - p[0][k];
            b[k] = p[2][k] - p[0][k];
            d[k] = p[3][k] - p[0][k];
        }
        double det = a[0] * (b[1] * d[2] - b[2] * d[1]) - a[1] * (b[0] * d[2] - b[2] * d[0])
                   + a[2] * (b[0] * d[1] - b[1] * d[0]);
        m->vol[c] = fabs(det) / 6.0;
        if (!(m->vol[c] > 0.0)) { *err = 2; orc_mesh_destroy(m); return NULL; }
    }

    /* faces: the face opposite vertex i is made of the other three vertices */
    for (int64_t c = 0; c < n_cells; ++c) {
        for (int i = 0; i < 4; ++i) {
            const double *q[3];
            int j = 0;
            for (int k = 0; k < 4; ++k)
                if (k != i) q[j++] = xyz + 3 * (int64_t)tet[4 * c + k];
            double u[3], w[3], s[3], xf[3];
            for (int k = 0; k < 3; ++k) {
                u[k] = q[1][k] - q[0][k];
                w[k] = q[2][k] - q[0][k];
                xf[k] = (q[0][k] + q[1][k] + q[2][k]) / 3.0;
            }
            s[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
            s[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
            s[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
            double A = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            /* orient outward: away from the cell centroid */
            double out = 0.0;
            for (int k = 0; k < 3; ++k) out += s[k] * (xf[k] - m->xc[3 * c + k]);
            double sg = out > 0.0 ? 1.0 : -1.0;
            m->area[4 * c + i] = A;
            for (int k = 0; k < 3; ++k) {
                m->nrm[12 * c + 3 * i + k] = sg * s[k] / A;
                m->xf[12 * c + 3 * i + k] = xf[k];
            }
        }
    }

    /* face matching by sorting the vertex triples */
    face_key *keys = (face_key *)malloc(sizeof(face_key) * 4 * n_cells);
    for (int64_t c = 0; c < n_cells; ++c) {
        for (int i = 0; i < 4; ++i) {
            int32_t v[3];
            int j = 0;
            for (int k = 0; k < 4; ++k)
                if (k != i) v[j++] = tet[4 * c + k];
            sort3(v);
            face_key *fk = &keys[4 * c + i];
            fk->a = v[0]; fk->b = v[1]; fk->c = v[2];
            fk->cell = (int32_t)c; fk->local = i;
        }
    }
    qsort(keys, 4 * n_cells, sizeof(face_key), cmp_face);
    m->n_boundary = 0;
    for (int64_t s = 0; s < 4 * n_cells;) {
        int64_t e = s + 1;
        while (e < 4 * n_cells && keys[e].a == keys[s].a && keys[e].b == keys[s].b
               && keys[e].c == keys[s].c) ++e;
        if (e - s == 1) {
            m->nb[4 * keys[s].cell + keys[s].local] = -1;
            m->n_boundary++;
        } else if (e - s == 2) {
            m->nb[4 * keys[s].cell + keys[s].local] = keys[s + 1].cell;
            m->nb[4 * keys[s + 1].cell + keys[s + 1].local] = keys[s].cell;
        } else {
            free(keys); *err = 3; orc_mesh_destroy(m); return NULL;
        }
        s = e;
    }
    free(keys);

    /* cells around each node */
    m->n2c_ptr = (int64_t *)calloc(n_nodes + 1, sizeof(int64_t));
    for (int64_t c = 0; c < n_cells; ++c)
        for (int i = 0; i < 4; ++i) m->n2c_ptr[tet[4 * c + i] + 1]++;
    for (int64_t n = 0; n < n_nodes; ++n) m->n2c_ptr[n + 1] += m->n2c_ptr[n];
    m->n2c = (int32_t *)malloc(sizeof(int32_t) * 4 * n_cells);
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * n_nodes);
    memcpy(fill, m->n2c_ptr, sizeof(int64_t) * n_nodes);
    for (int64_t c = 0; c < n_cells; ++c)
        for (int i = 0; i < 4; ++i) m->n2c[fill[tet[4 * c + i]]++] = (int32_t)c;
    free(fill);
    return m;
}

int64_t orc_mesh_n_boundary_faces(const orc_mesh *m) { return m->n_boundary; }

void orc_mesh_cell_info(const orc_mesh *m, double *centroid, double *volume,
                        int32_t *neighbour) {
    if (centroid) memcpy(centroid, m->xc, sizeof(double) * 3 * m->n_cells);
    if (volume) memcpy(volume, m->vol, sizeof(double) * m->n_cells);
    if (neighbour) memcpy(neighbour, m->nb, sizeof(int32_t) * 4 * m->n_cells);
}

/* S1: inverse-distance weighted node values. */
void orc_node_values(const orc_mesh *m, const double *v, double *vn) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < m->n_nodes; ++n) {
        double num = 0.0, den = 0.0;
        for (int64_t k = m->n2c_ptr[n]; k < m->n2c_ptr[n + 1]; ++k) {
            int32_t c = m->n2c[k];
            double dx = m->xyz[3 * n] - m->xc[3 * c];
            double dy = m->xyz[3 * n + 1] - m->xc[3 * c + 1];
            double dz = m->xyz[3 * n + 2] - m->xc[3 * c + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            num += v[c] / d;
            den += 1.0 / d;
        }
        vn[n] = den > 0.0 ? num / den : 0.0;
    }
}

/* S2: face values from the three face vertices, then Gauss-Green. */
void orc_cell_gradients(const orc_mesh *m, const double *vn, double *grad) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m->n_cells; ++c) {
        double g[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 4; ++i) {
            double vf = 0.0;
            for (int k = 0; k < 4; ++k)
                if (k != i) vf += vn[m->tet[4 * c + k]];
            vf /= 3.0;
            for (int k = 0; k < 3; ++k)
                g[k] += vf * m->area[4 * c + i] * m->nrm[12 * c + 3 * i + k];
        }
        for (int k = 0; k < 3; ++k) grad[3 * c + k] = g[k] / m->vol[c];
    }
}

static double dist3(const double *a, const double *b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* S3 and the sum of Eq. 7, divided by the cell volume. */
void orc_diffusion(const orc_mesh *m, const double *D, const double *v, double *out) {
    double *vn = (double *)malloc(sizeof(double) * m->n_nodes);
    double *grad = (double *)malloc(sizeof(double) * 3 * m->n_cells);
    orc_node_values(m, v, vn);
    orc_cell_gradients(m, vn, grad);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m->n_cells; ++c) {
        double sum = 0.0;
        for (int i = 0; i < 4; ++i) {
            int32_t c2 = m->nb[4 * c + i];
            if (c2 < 0) continue;                       /* zero-flux boundary face */
            const double *x1 = m->xc + 3 * c, *x2 = m->xc + 3 * (int64_t)c2;
            const double *xf = m->xf + 12 * c + 3 * i;
            const double *n = m->nrm + 12 * c + 3 * i;
            double r1 = dist3(x1, xf), r2 = dist3(x2, xf);
            double a1 = r2 / (r1 + r2), a2 = 1.0 - a1;
            double d = dist3(x1, x2);
            double e[3], gbar[3], gf[3];
            for (int k = 0; k < 3; ++k) {
                e[k] = (x1[k] - x2[k]) / d;
                gbar[k] = a1 * grad[3 * c + k] + a2 * grad[3 * (int64_t)c2 + k];
            }
            double gbar_e = gbar[0] * e[0] + gbar[1] * e[1] + gbar[2] * e[2];
            double corr = (v[c] - v[c2]) / d - gbar_e;
            for (int k = 0; k < 3; ++k) gf[k] = gbar[k] + corr * e[k];
            /* face tensor and flux A_f (D_f grad v_f) . n_f */
            double flux = 0.0;
            for (int r = 0; r < 3; ++r) {
                double Dg = 0.0;
                for (int k = 0; k < 3; ++k) {
                    double Df = a1 * D[9 * c + 3 * r + k] + a2 * D[9 * (int64_t)c2 + 3 * r + k];
                    Dg += Df * gf[k];
                }
                flux += Dg * n[r];
            }
            sum += m->area[4 * c + i] * flux;
        }
        out[c] = sum / m->vol[c];
    }
    free(vn);
    free(grad);
}

/* The two-point part alone: grad v_f replaced by [(v_c1 - v_c2)/d] e. Its
 * volume-weighted matrix is symmetric; used as a check of the face tensors. */
void orc_diffusion_twopoint(const orc_mesh *m, const double *D, const double *v, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < m->n_cells; ++c) {
        double sum = 0.0;
        for (int i = 0; i < 4; ++i) {
            int32_t c2 = m->nb[4 * c + i];
            if (c2 < 0) continue;
            const double *x1 = m->xc + 3 * c, *x2 = m->xc + 3 * (int64_t)c2;
            const double *xf = m->xf + 12 * c + 3 * i;
            const double *n = m->nrm + 12 * c + 3 * i;
            double r1 = dist3(x1, xf), r2 = dist3(x2, xf);
            double a1 = r2 / (r1 + r2), a2 = 1.0 - a1;
            double d = dist3(x1, x2);
            double e[3];
            for (int k = 0; k < 3; ++k) e[k] = (x1[k] - x2[k]) / d;
            double s = (v[c] - v[c2]) / d;
            double flux = 0.0;
            for (int r = 0; r < 3; ++r) {
                double Dg = 0.0;
                for (int k = 0; k < 3; ++k)
                    Dg += (a1 * D[9 * c + 3 * r + k] + a2 * D[9 * (int64_t)c2 + 3 * r + k]) * s * e[k];
                flux += Dg * n[r];
            }
            sum += m->area[4 * c + i] * flux;
        }
        out[c] = sum / m->vol[c];
    }
}

/* Eqs. 2-3: D = A diag(D_l, D_t, D_t) A^T, A = [fibre, sheet, normal] column-wise.
 * The sheet direction is any unit vector orthogonal to the fibre (the
 * transverse conductivities are equal, Table 2). */
void orc_conductivity(const double *fibre, double D_l, double D_t, double *D) {
    double f[3] = {fibre[0], fibre[1], fibre[2]};
    double nf = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int k = 0; k < 3; ++k) f[k] /= nf;
    double ax[3] = {0.0, 0.0, 0.0};
    int imin = 0;
    for (int k = 1; k < 3; ++k) if (fabs(f[k]) < fabs(f[imin])) imin = k;
    ax[imin] = 1.0;
    double s[3] = {f[1] * ax[2] - f[2] * ax[1], f[2] * ax[0] - f[0] * ax[2], f[0] * ax[1] - f[1] * ax[0]};
    double ns = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int k = 0; k < 3; ++k) s[k] /= ns;
    double n[3] = {f[1] * s[2] - f[2] * s[1], f[2] * s[0] - f[0] * s[2], f[0] * s[1] - f[1] * s[0]};
    double A[3][3], Dhat[3] = {D_l, D_t, D_t};
    for (int r = 0; r < 3; ++r) { A[r][0] = f[r]; A[r][1] = s[r]; A[r][2] = n[r]; }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += A[r][k] * Dhat[k] * A[c][k];
            D[3 * r + c] = acc;
        }
}
