// Host planner of the monodomain finite-volume step (see planner.h).
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

namespace ep {

namespace {

struct V3 {
    double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

inline V3 node(const std::vector<double> &xyz, int64_t n) { return {xyz[3 * n], xyz[3 * n + 1], xyz[3 * n + 2]}; }

// Geometry of one tetrahedron: centroid, volume, outward area vectors of the
// faces opposite each vertex and their centroids, and the gradient weights
// b_k = -S_k / (3 V) of the Gauss-Green gradient of the vertex-averaged face
// values (sum_k b_k v_k equals (1/V) sum_faces v_f S_f with v_f the mean of the
// face's three vertex values).
struct TetGeom {
    V3 c;
    double vol;
    V3 S[4], xf[4], b[4];
};

TetGeom tet_geom(const std::vector<double> &xyz, const int32_t *t) {
    TetGeom g;
    V3 p[4];
    for (int k = 0; k < 4; ++k) p[k] = node(xyz, t[k]);
    g.c = 0.25 * (p[0] + p[1] + p[2] + p[3]);
    g.vol = dot(cross(p[1] - p[0], p[2] - p[0]), p[3] - p[0]) / 6.0;
    for (int k = 0; k < 4; ++k) {
        const V3 &a = p[(k + 1) & 3], &b = p[(k + 2) & 3], &d = p[(k + 3) & 3];
        V3 s = 0.5 * cross(b - a, d - a);
        V3 xf = (1.0 / 3.0) * (a + b + d);
        if (dot(s, xf - p[k]) < 0.0) s = -1.0 * s;
        g.S[k] = s;
        g.xf[k] = xf;
        g.b[k] = (-1.0 / (3.0 * g.vol)) * s;
    }
    return g;
}

// Geometry of a shell triangle in the same form: area in `vol`, the
// in-plane outward edge normals times edge lengths in S (edge k opposite
// node k), edge midpoints in xf, b_k = -S_k / (2 A) (Gauss-Green of the
// edge-averaged node values); slot 3 unused.
TetGeom tri_geom(const std::vector<double> &xyz, const int32_t *t) {
    TetGeom g;
    V3 p[3];
    for (int k = 0; k < 3; ++k) p[k] = node(xyz, t[k]);
    g.c = (1.0 / 3.0) * (p[0] + p[1] + p[2]);
    const V3 w = cross(p[1] - p[0], p[2] - p[0]);
    const double nw = norm(w);
    const V3 un = (1.0 / nw) * w;
    g.vol = 0.5 * nw;
    for (int k = 0; k < 3; ++k) {
        const V3 &a = p[(k + 1) % 3], &b = p[(k + 2) % 3];
        const V3 tv = b - a, mid = 0.5 * (a + b);
        V3 n = cross(tv, un);
        n = (1.0 / norm(n)) * n;
        if (dot(n, mid - p[k]) < 0.0) n = -1.0 * n;
        g.S[k] = norm(tv) * n;
        g.xf[k] = mid;
        g.b[k] = (-1.0 / (2.0 * g.vol)) * g.S[k];
    }
    g.S[3] = g.xf[3] = g.b[3] = V3{0.0, 0.0, 0.0};
    return g;
}

TetGeom cell_geom(const HostMesh &m, int64_t c) {
    const int32_t *t = &m.tet[4 * c];
    return (!m.kind.empty() && m.kind[c]) ? tri_geom(m.xyz, t) : tet_geom(m.xyz, t);
}

void tensor(const HostMesh &m, const ep_params *p, int64_t c, double D[9]) {
    const ep_cell_params &cp = p->sets[m.pset[c]];
    if (m.fibre.empty()) {
        for (int i = 0; i < 9; ++i) D[i] = (i % 4 == 0) ? cp.D_l : 0.0;
        return;
    }
    V3 f{m.fibre[3 * c], m.fibre[3 * c + 1], m.fibre[3 * c + 2]};
    f = (1.0 / norm(f)) * f;
    const double ff[3] = {f.x, f.y, f.z};
    // transversely isotropic: D = D_t I + (D_l - D_t) f f^T
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) D[3 * r + k] = (r == k ? cp.D_t : 0.0) + (cp.D_l - cp.D_t) * ff[r] * ff[k];
}

struct FaceRec {
    int32_t b, c;      // the two larger vertex ids (the smallest is the bucket)
    int32_t cell;
    int8_t local;
};

}  // namespace

int build_mesh(const ep_mesh_desc *d, HostMesh *m, std::string *err) {
    const int64_t NT = d->n_cells, NS = d->n_tris, N = NT + NS, NN = d->n_nodes;
    if (d->index_width != 0 && d->index_width != 16 && d->index_width != 32) {
        *err = "mesh: index_width must be 0 (automatic), 16 or 32";
        return EP_EINVAL;
    }
    m->index_width = d->index_width;
    if (NT < 0 || NS < 0 || N <= 0 || NN <= 0 || !d->xyz || (NT > 0 && !d->tet) || (NS > 0 && !d->tri)) {
        *err = "mesh: empty mesh or NULL xyz/tet/tri";
        return EP_EINVAL;
    }
    if (N >= (int64_t(1) << 31) || NN >= (int64_t(1) << 31)) {
        *err = "mesh: more than 2^31-1 cells or nodes";
        return EP_EINVAL;
    }
    // cells: the tets, then the shell triangles (slot 3 repeats the first node)
    std::vector<int32_t> tet(4 * N);
    std::vector<uint8_t> kind0(N, 0);
    if (NT > 0) std::copy(d->tet, d->tet + 4 * NT, tet.begin());
    for (int64_t s = 0; s < NS; ++s) {
        for (int k = 0; k < 3; ++k) tet[4 * (NT + s) + k] = d->tri[3 * s + k];
        tet[4 * (NT + s) + 3] = d->tri[3 * s];
        kind0[NT + s] = 1;
    }
    for (int64_t i = 0; i < 4 * N; ++i)
        if (tet[i] < 0 || tet[i] >= NN) {
            *err = "mesh: node index out of range in cell " + std::to_string(i / 4);
            return EP_EMESH;
        }
    std::vector<double> xyz0(d->xyz, d->xyz + 3 * NN);
    // orientation and degeneracy
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t n = 0; n < NN; ++n)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], xyz0[3 * n + k]);
            hi[k] = std::max(hi[k], xyz0[3 * n + k]);
        }
    int bad = -1;
#pragma omp parallel for schedule(static)
    for (int64_t c = NT; c < N; ++c) {   // triangles: non-zero area
        const int32_t *t = &tet[4 * c];
        V3 e1 = node(xyz0, t[1]) - node(xyz0, t[0]), e2 = node(xyz0, t[2]) - node(xyz0, t[0]);
        double l = std::max(norm(e1), norm(e2));
        if (!(norm(cross(e1, e2)) > 1e-12 * l * l)) {
#pragma omp critical
            bad = (bad < 0) ? int(c) : std::min(bad, int(c));
        }
    }
    if (bad >= 0) {
        *err = "mesh: degenerate (zero-area) triangle " + std::to_string(bad - NT);
        return EP_EMESH;
    }
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < NT; ++c) {
        int32_t *t = &tet[4 * c];
        V3 p0 = node(xyz0, t[0]), p1 = node(xyz0, t[1]), p2 = node(xyz0, t[2]), p3 = node(xyz0, t[3]);
        V3 e1 = p1 - p0, e2 = p2 - p0, e3 = p3 - p0;
        double det = dot(cross(e1, e2), e3);
        double l = std::max(norm(e1), std::max(norm(e2), norm(e3)));
        if (!(std::fabs(det) > 1e-12 * l * l * l)) {
#pragma omp critical
            bad = (bad < 0) ? int(c) : std::min(bad, int(c));
        }
        if (det < 0) std::swap(t[2], t[3]);
    }
    if (bad >= 0) {
        *err = "mesh: degenerate (zero-volume) tetrahedron " + std::to_string(bad);
        return EP_EMESH;
    }
    // faces: bucket by smallest vertex, then sort each bucket
    std::vector<int64_t> bptr(NN + 1, 0);
    for (int64_t c = 0; c < NT; ++c)
        for (int k = 0; k < 4; ++k) {
            int32_t a = INT32_MAX;
            for (int j = 0; j < 4; ++j)
                if (j != k) a = std::min(a, tet[4 * c + j]);
            bptr[a + 1]++;
        }
    for (int64_t n = 0; n < NN; ++n) bptr[n + 1] += bptr[n];
    std::vector<FaceRec> recs(4 * NT);
    {
        std::vector<int64_t> fill(bptr.begin(), bptr.end() - 1);
        for (int64_t c = 0; c < NT; ++c)
            for (int k = 0; k < 4; ++k) {
                int32_t v[3];
                int j = 0;
                for (int i = 0; i < 4; ++i)
                    if (i != k) v[j++] = tet[4 * c + i];
                std::sort(v, v + 3);
                recs[fill[v[0]]++] = FaceRec{v[1], v[2], int32_t(c), int8_t(k)};
            }
    }
    std::vector<int32_t> nbr0(4 * N, -1);
    int64_t n_int = 0;
    bool nonmanifold = false;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : n_int)
    for (int64_t a = 0; a < NN; ++a) {
        auto beg = recs.begin() + bptr[a], end = recs.begin() + bptr[a + 1];
        std::sort(beg, end, [](const FaceRec &x, const FaceRec &y) {
            if (x.b != y.b) return x.b < y.b;
            if (x.c != y.c) return x.c < y.c;
            return x.cell < y.cell;
        });
        for (auto s = beg; s != end;) {
            auto e = s + 1;
            while (e != end && e->b == s->b && e->c == s->c) ++e;
            if (e - s == 2) {
                nbr0[4 * int64_t(s->cell) + s->local] = (s + 1)->cell;
                nbr0[4 * int64_t((s + 1)->cell) + (s + 1)->local] = s->cell;
                ++n_int;
            } else if (e - s > 2) {
                nonmanifold = true;
            }
            s = e;
        }
    }
    if (nonmanifold) {
        *err = "mesh: a face is shared by more than two tetrahedra";
        return EP_EMESH;
    }
    recs.clear();
    recs.shrink_to_fit();
    // shell edges: the edge opposite node k of a triangle, matched by its sorted node pair
    {
        struct EdgeRec {
            int32_t a, b, cell;
            int8_t local;
        };
        std::vector<EdgeRec> er;
        er.reserve(3 * NS);
        for (int64_t c = NT; c < N; ++c)
            for (int k = 0; k < 3; ++k) {
                int32_t a = tet[4 * c + (k + 1) % 3], b = tet[4 * c + (k + 2) % 3];
                if (a > b) std::swap(a, b);
                er.push_back(EdgeRec{a, b, int32_t(c), int8_t(k)});
            }
        std::sort(er.begin(), er.end(), [](const EdgeRec &x, const EdgeRec &y) {
            if (x.a != y.a) return x.a < y.a;
            if (x.b != y.b) return x.b < y.b;
            return x.cell < y.cell;
        });
        for (size_t i = 0; i < er.size();) {
            size_t e = i + 1;
            while (e < er.size() && er[e].a == er[i].a && er[e].b == er[i].b) ++e;
            if (e - i == 2) {
                nbr0[4 * int64_t(er[i].cell) + er[i].local] = er[i + 1].cell;
                nbr0[4 * int64_t(er[i + 1].cell) + er[i + 1].local] = er[i].cell;
                ++n_int;
            } else if (e - i > 2) {
                *err = "mesh: an edge is shared by more than two shell triangles";
                return EP_EMESH;
            }
            i = e;
        }
    }

    // model of each cell
    std::vector<uint8_t> model0(N, EP_TP06);
    if (d->cell_model)
        for (int64_t c = 0; c < N; ++c) {
            if (d->cell_model[c] >= EP_N_MODELS) {
                *err = "mesh: unknown cell model in cell " + std::to_string(c);
                return EP_EINVAL;
            }
            model0[c] = d->cell_model[c];
        }

    // reverse Cuthill-McKee on the face-adjacency graph
    auto degree = [&](int64_t c) {
        int dg = 0;
        for (int k = 0; k < 4; ++k) dg += nbr0[4 * c + k] >= 0;
        return dg;
    };
    std::vector<int32_t> order;
    order.reserve(N);
    std::vector<int32_t> level(N, -1);
    std::vector<char> visited(N, 0);
    // BFS over the component of s; q receives the visit order and level[] the
    // distance of each visited cell (reset with clear_levels)
    auto bfs = [&](int32_t s, std::vector<int32_t> &q) {
        q.clear();
        q.push_back(s);
        level[s] = 0;
        for (size_t h = 0; h < q.size(); ++h) {
            int32_t u = q[h];
            for (int k = 0; k < 4; ++k) {
                int32_t v = nbr0[4 * int64_t(u) + k];
                if (v >= 0 && level[v] < 0) {
                    level[v] = level[u] + 1;
                    q.push_back(v);
                }
            }
        }
        return level[q.back()];
    };
    auto clear_levels = [&](const std::vector<int32_t> &q) {
        for (int32_t u : q) level[u] = -1;
    };
    std::vector<int32_t> q;
    for (int64_t root = 0; root < N; ++root) {
        if (visited[root]) continue;
        // pseudo-peripheral start: restart from a minimum-degree cell of the
        // last BFS level while the eccentricity grows
        int32_t s = int32_t(root);
        int ecc = bfs(s, q);
        for (int it = 0; it < 4; ++it) {
            int32_t best = q.back();
            int bd = 5;
            for (auto r = q.rbegin(); r != q.rend() && level[*r] == ecc; ++r) {
                int dg = degree(*r);
                if (dg < bd || (dg == bd && *r < best)) {
                    bd = dg;
                    best = *r;
                }
            }
            clear_levels(q);
            int e2 = bfs(best, q);
            if (e2 <= ecc) break;
            s = best;
            ecc = e2;
        }
        clear_levels(q);
        // Cuthill-McKee from s
        size_t head = order.size();
        order.push_back(s);
        visited[s] = 1;
        for (size_t h = head; h < order.size(); ++h) {
            int32_t u = order[h];
            int32_t nb[4];
            int cnt = 0;
            for (int k = 0; k < 4; ++k) {
                int32_t v = nbr0[4 * int64_t(u) + k];
                if (v >= 0 && !visited[v]) {
                    nb[cnt++] = v;
                    visited[v] = 1;
                }
            }
            std::sort(nb, nb + cnt, [&](int32_t x, int32_t y) {
                int dx = degree(x), dy = degree(y);
                return dx != dy ? dx < dy : x < y;
            });
            for (int i = 0; i < cnt; ++i) order.push_back(nb[i]);
        }
    }
    std::reverse(order.begin(), order.end());
    // group by cell model, keeping the RCM order inside each group
    std::stable_partition(order.begin(), order.end(), [&](int32_t c) { return model0[c] == EP_TP06; });
    auto mid = std::find_if(order.begin(), order.end(), [&](int32_t c) { return model0[c] != EP_TP06; });
    std::stable_partition(mid, order.end(), [&](int32_t c) { return model0[c] == EP_CRN; });

    m->n_cells = N;
    m->cell_new2old = order;
    std::vector<int32_t> old2new(N);
    for (int64_t i = 0; i < N; ++i) old2new[order[i]] = int32_t(i);
    // node order of first appearance
    std::vector<int32_t> nold2new(NN, -1);
    m->node_new2old.clear();
    m->node_new2old.reserve(NN);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < 4; ++k) {
            int32_t v = tet[4 * int64_t(order[i]) + k];
            if (nold2new[v] < 0) {
                nold2new[v] = int32_t(m->node_new2old.size());
                m->node_new2old.push_back(v);
            }
        }
    for (int64_t v = 0; v < NN; ++v)
        if (nold2new[v] < 0) {
            nold2new[v] = int32_t(m->node_new2old.size());
            m->node_new2old.push_back(int32_t(v));
        }
    m->n_nodes = NN;
    m->xyz.resize(3 * NN);
    for (int64_t n = 0; n < NN; ++n)
        for (int k = 0; k < 3; ++k) m->xyz[3 * n + k] = xyz0[3 * int64_t(m->node_new2old[n]) + k];
    m->tet.resize(4 * N);
    m->kind.resize(N);
    m->nbr.resize(4 * N);
    m->opp.resize(4 * N);
    m->model.resize(N);
    m->pset.resize(N);
    m->smask.resize(N);
    if (d->fibre) m->fibre.resize(3 * N);
    else m->fibre.clear();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t o = order[i];
        for (int k = 0; k < 4; ++k) {
            m->tet[4 * i + k] = nold2new[tet[4 * o + k]];
            int32_t nb = nbr0[4 * o + k];
            m->nbr[4 * i + k] = nb < 0 ? -1 : old2new[nb];
        }
        m->model[i] = model0[o];
        m->kind[i] = kind0[o];
        m->pset[i] = d->param_set ? d->param_set[o] : 0;
        m->smask[i] = d->stim_mask ? d->stim_mask[o] : 0;
        if (d->fibre)
            for (int k = 0; k < 3; ++k) m->fibre[3 * i + k] = d->fibre[3 * o + k];
    }
    for (int64_t i = 0; i < N; ++i)
        if (!m->fibre.empty()) {
            double f2 = m->fibre[3 * i] * m->fibre[3 * i] + m->fibre[3 * i + 1] * m->fibre[3 * i + 1] +
                        m->fibre[3 * i + 2] * m->fibre[3 * i + 2];
            if (!(f2 > 0.0) || !std::isfinite(f2)) {
                *err = "mesh: zero or non-finite fibre direction in cell " + std::to_string(m->cell_new2old[i]);
                return EP_EINVAL;
            }
        }
    // neighbour's vertex opposite each interior face (edge, for a triangle)
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const int nv = m->kind[i] ? 3 : 4;
        for (int k = 0; k < 4; ++k) {
            int32_t nb = m->nbr[4 * i + k];
            int32_t o = -1;
            if (nb >= 0) {
                const int nvb = m->kind[nb] ? 3 : 4;
                for (int j = 0; j < nvb; ++j) {
                    int32_t v = m->tet[4 * int64_t(nb) + j];
                    bool in_face = false;
                    for (int l = 0; l < nv; ++l)
                        if (l != k && m->tet[4 * i + l] == v) in_face = true;
                    if (!in_face) o = v;
                }
            }
            m->opp[4 * i + k] = o;
        }
    }
    m->n_interior_faces = n_int;
    for (int mdl = 0; mdl <= EP_N_MODELS; ++mdl) m->model_off[mdl] = 0;
    for (int64_t i = 0; i < N; ++i) m->model_off[m->model[i] + 1]++;
    for (int mdl = 0; mdl < EP_N_MODELS; ++mdl) m->model_off[mdl + 1] += m->model_off[mdl];
    // node -> cell incidence, cells ascending
    m->n2c_ptr.assign(NN + 1, 0);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < (m->kind[i] ? 3 : 4); ++k) m->n2c_ptr[m->tet[4 * i + k] + 1]++;
    for (int64_t n = 0; n < NN; ++n) m->n2c_ptr[n + 1] += m->n2c_ptr[n];
    m->n2c.resize(m->n2c_ptr[NN]);
    {
        std::vector<int64_t> fill(m->n2c_ptr.begin(), m->n2c_ptr.end() - 1);
        for (int64_t i = 0; i < N; ++i)
            for (int k = 0; k < (m->kind[i] ? 3 : 4); ++k) m->n2c[fill[m->tet[4 * i + k]]++] = int32_t(i);
    }
    return EP_OK;
}

int build_coeffs(const HostMesh &m, const ep_params *p, Coeffs *cf, std::string *err) {
    const int64_t N = m.n_cells;
    for (int64_t i = 0; i < N; ++i)
        if (m.pset[i] >= p->n_sets) {
            *err = "params: cell " + std::to_string(m.cell_new2old[i]) + " uses parameter set " +
                   std::to_string(m.pset[i]) + " but only " + std::to_string(p->n_sets) + " are given";
            return EP_EINVAL;
        }
    cf->wa.assign(4 * N, 0.0);
    cf->wb.assign(4 * N, 0.0);
    cf->q.assign(4 * N, 0.0);
    cf->nw.assign(m.n2c.size(), 0.0);
    double gmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : gmax)
    for (int64_t c = 0; c < N; ++c) {
        const int32_t *tc = &m.tet[4 * c];
        const bool tri = !m.kind.empty() && m.kind[c];
        const int nv = tri ? 3 : 4;
        TetGeom g = cell_geom(m, c);
        double Dc[9];
        tensor(m, p, c, Dc);
        double wa[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0}, q[4] = {0, 0, 0, 0};
        for (int k = 0; k < nv; ++k) {
            int32_t nb = m.nbr[4 * c + k];
            if (nb < 0) continue;  // zero-flux boundary face
            const int32_t *tn = &m.tet[4 * int64_t(nb)];
            TetGeom gn = cell_geom(m, nb);
            double Dn[9];
            tensor(m, p, nb, Dn);
            const V3 xf = g.xf[k];
            double r1 = norm(g.c - xf), r2 = norm(gn.c - xf);
            double alpha = r2 / (r1 + r2);
            V3 dvec = g.c - gn.c;
            double dist = norm(dvec);
            V3 e = (1.0 / dist) * dvec;
            // a = D_f S (face tensor times outward area vector)
            double Df[9];
            for (int i = 0; i < 9; ++i) Df[i] = alpha * Dc[i] + (1.0 - alpha) * Dn[i];
            V3 S = g.S[k];
            if (tri) {
                // the two triangles of an edge may lie in different planes: both use the
                // normalised mean of their outward normals (conservative edge flux)
                int k2 = 0;
                for (int l = 0; l < 3; ++l)
                    if (m.nbr[4 * int64_t(nb) + l] == int32_t(c)) k2 = l;
                const double L = norm(S);
                V3 nrm = (1.0 / L) * S - (1.0 / norm(gn.S[k2])) * gn.S[k2];
                S = (L / norm(nrm)) * nrm;
            }
            V3 a{Df[0] * S.x + Df[1] * S.y + Df[2] * S.z, Df[3] * S.x + Df[4] * S.y + Df[5] * S.z,
                 Df[6] * S.x + Df[7] * S.y + Df[8] * S.z};
            double ae = dot(a, e);
            V3 pvec = a - ae * e;  // acts on the interpolated face gradient
            double qq = ae / dist; // acts on V_c - V_nb
            for (int j = 0; j < nv; ++j) wa[j] += alpha * dot(pvec, g.b[j]);
            const int nvn = (!m.kind.empty() && m.kind[nb]) ? 3 : 4;
            for (int j = 0; j < nvn; ++j) {
                double coef = (1.0 - alpha) * dot(pvec, gn.b[j]);
                int32_t v = tn[j];
                int slot = -1;
                for (int l = 0; l < nv; ++l)
                    if (tc[l] == v) slot = l;
                if (slot >= 0) wa[slot] += coef;
                else wb[k] += coef;
            }
            q[k] = -qq;
        }
        double inv = 1.0 / g.vol, rs = 0.0;
        for (int k = 0; k < 4; ++k) {
            cf->wa[4 * c + k] = wa[k] * inv;
            cf->wb[4 * c + k] = wb[k] * inv;
            cf->q[4 * c + k] = q[k] * inv;
            rs += std::fabs(wa[k] * inv) + std::fabs(wb[k] * inv) + 2.0 * std::fabs(q[k] * inv);
        }
        gmax = std::max(gmax, rs);
    }
    cf->gershgorin = gmax;
    // inverse-distance node weights, normalised per node
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < m.n_nodes; ++n) {
        V3 xn = node(m.xyz, n);
        double s = 0.0;
        for (int64_t j = m.n2c_ptr[n]; j < m.n2c_ptr[n + 1]; ++j) {
            const int64_t cc = m.n2c[j];
            const int32_t *t = &m.tet[4 * cc];
            V3 xc = (!m.kind.empty() && m.kind[cc])
                        ? (1.0 / 3.0) * (node(m.xyz, t[0]) + node(m.xyz, t[1]) + node(m.xyz, t[2]))
                        : 0.25 * (node(m.xyz, t[0]) + node(m.xyz, t[1]) + node(m.xyz, t[2]) + node(m.xyz, t[3]));
            double w = 1.0 / norm(xn - xc);
            cf->nw[j] = w;
            s += w;
        }
        for (int64_t j = m.n2c_ptr[n]; j < m.n2c_ptr[n + 1]; ++j) cf->nw[j] /= s;
    }
    return EP_OK;
}

double power_radius(const HostMesh &m, const Coeffs &cf, int iters) {
    const int64_t N = m.n_cells;
    std::vector<double> x(N), y(N), vn(m.n_nodes);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (int64_t i = 0; i < N; ++i) {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        x[i] = double(st >> 11) / double(1ull << 53) - 0.5;
    }
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < m.n_nodes; ++n) {
            double s = 0.0;
            for (int64_t j = m.n2c_ptr[n]; j < m.n2c_ptr[n + 1]; ++j) s += cf.nw[j] * x[m.n2c[j]];
            vn[n] = s;
        }
        double num = 0.0, den = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : num, den)
        for (int64_t c = 0; c < N; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) {
                s += cf.wa[4 * c + k] * vn[m.tet[4 * c + k]];
                if (m.opp[4 * c + k] >= 0) s += cf.wb[4 * c + k] * vn[m.opp[4 * c + k]];
                int32_t nb = m.nbr[4 * c + k];
                if (nb >= 0) s += cf.q[4 * c + k] * (x[nb] - x[c]);
            }
            y[c] = s;
            num += s * s;
            den += x[c] * x[c];
        }
        lam = std::sqrt(num / den);
        double inv = 1.0 / std::sqrt(num);
        for (int64_t c = 0; c < N; ++c) x[c] = y[c] * inv;
    }
    return lam;
}

void cell_gather_indices(const HostMesh &m, int64_t c, int32_t na[4], int32_t nb[4], int32_t nc[4]) {
    const int32_t *t = &m.tet[4 * c];
    for (int k = 0; k < 4; ++k) {
        na[k] = t[k];
        nb[k] = m.opp[4 * c + k] >= 0 ? m.opp[4 * c + k] : t[0];
        nc[k] = m.nbr[4 * c + k] >= 0 ? m.nbr[4 * c + k] : int32_t(c);
    }
}

// 16-bit form of the ELL entries (see Sell), if every slice's offsets fit.
static bool build_col16(Sell *s) {
    const int64_t ns = int64_t(s->slice_ptr.size()) - 1;
    s->cbase.assign(ns, 0);
    s->col16.assign(s->col.size(), 0);
    for (int64_t sl = 0; sl < ns; ++sl) {
        const int64_t b = s->slice_ptr[sl], e = s->slice_ptr[sl + 1];
        if (b == e) continue;
        int32_t lo = s->col[b], hi = s->col[b];
        for (int64_t k = b; k < e; ++k) lo = std::min(lo, s->col[k]), hi = std::max(hi, s->col[k]);
        if (int64_t(hi) - lo > 65535) return false;
        s->cbase[sl] = lo;
        for (int64_t k = b; k < e; ++k) s->col16[k] = uint16_t(s->col[k] - lo);
    }
    return true;
}

// 16-bit form of the cells' gather indices (see Sell), if every offset fits.
static bool build_idx16(const HostMesh &m, Sell *s) {
    const int64_t N = m.n_cells, NN = m.n_nodes;
    const int64_t nblk = (N + 255) / 256;
    s->nbase.assign(nblk, 0);
    s->cidx16.assign(8 * N, 0);
    s->nbr16.assign(4 * N, 0);
    for (int64_t blk = 0; blk < nblk; ++blk) {
        const int64_t c0 = 256 * blk, c1 = std::min(N, c0 + 256);
        int32_t lo = int32_t(NN), hi = 0;
        int32_t na[4], nb[4], nc[4];
        for (int64_t c = c0; c < c1; ++c) {
            cell_gather_indices(m, c, na, nb, nc);
            for (int k = 0; k < 4; ++k) {
                lo = std::min({lo, na[k], nb[k]});
                hi = std::max({hi, na[k], nb[k]});
            }
        }
        if (int64_t(hi) - lo > 65535) return false;
        s->nbase[blk] = lo;
        for (int64_t c = c0; c < c1; ++c) {
            cell_gather_indices(m, c, na, nb, nc);
            for (int k = 0; k < 4; ++k) {
                s->cidx16[8 * c + k] = uint16_t(na[k] - lo);
                s->cidx16[8 * c + 4 + k] = uint16_t(nb[k] - lo);
                const int64_t d = int64_t(nc[k]) - c;
                if (d < -32768 || d > 32767) return false;
                s->nbr16[4 * c + k] = int16_t(d);
            }
        }
    }
    return true;
}

void build_sell(const HostMesh &m, Sell *s) {
    const int64_t NN = m.n_nodes;
    const int64_t ns = (NN + 31) / 32;
    s->slice_ptr.assign(ns + 1, 0);
    for (int64_t sl = 0; sl < ns; ++sl) {
        int64_t len = 0;
        for (int64_t n = sl * 32; n < std::min(NN, sl * 32 + 32); ++n)
            len = std::max(len, m.n2c_ptr[n + 1] - m.n2c_ptr[n]);
        s->slice_ptr[sl + 1] = s->slice_ptr[sl] + 32 * len;
    }
    s->col.assign(s->slice_ptr[ns], 0);
    s->src.assign(s->slice_ptr[ns], -1);
#pragma omp parallel for schedule(static)
    for (int64_t sl = 0; sl < ns; ++sl) {
        int64_t len = (s->slice_ptr[sl + 1] - s->slice_ptr[sl]) / 32;
        // pads repeat a cell of the slice itself, so that they stay inside its window of cells
        int32_t slice_pad = 0;
        for (int64_t n = sl * 32; n < std::min(NN, sl * 32 + 32); ++n)
            if (m.n2c_ptr[n + 1] > m.n2c_ptr[n]) {
                slice_pad = m.n2c[m.n2c_ptr[n]];
                break;
            }
        for (int lane = 0; lane < 32; ++lane) {
            int64_t n = sl * 32 + lane;
            int64_t b = n < NN ? m.n2c_ptr[n] : 0, e = n < NN ? m.n2c_ptr[n + 1] : 0;
            int32_t pad_col = (e > b) ? m.n2c[b] : slice_pad;
            for (int64_t k = 0; k < len; ++k) {
                int64_t at = s->slice_ptr[sl] + k * 32 + lane;
                if (b + k < e) {
                    s->col[at] = m.n2c[b + k];
                    s->src[at] = b + k;
                } else {
                    s->col[at] = pad_col;
                    s->src[at] = -1;
                }
            }
        }
    }
    s->idx16 = m.index_width != 32 && build_idx16(m, s);
    if (!s->idx16) {
        s->cidx16.clear();
        s->nbr16.clear();
        s->nbase.clear();
    }
    // the 16-bit node table only on request: it moves 2 bytes less per entry, but on the B300 its
    // node pass ran slower than the 32-bit one (18.5 against 14.3 us on the 1.2M-cell crop)
    s->col16ok = m.index_width == 16 && build_col16(s);
    if (!s->col16ok) {
        s->col16.clear();
        s->cbase.clear();
    }
}

}  // namespace ep
