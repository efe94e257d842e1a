// Host planning of a conduction graph (see graph_plan.h).
#include "graph_plan.h"
#include "devtypes.h"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace ep {

namespace {

struct P3 {
    double x, y, z;
};

P3 centroid(const HostMesh &m, int64_t c) {
    P3 r{0, 0, 0};
    const int nv = (!m.kind.empty() && m.kind[c]) ? 3 : 4;   // a shell triangle or a tetrahedron
    for (int k = 0; k < nv; ++k) {
        const int64_t v = m.tet[4 * c + k];
        r.x += m.xyz[3 * v] / nv;
        r.y += m.xyz[3 * v + 1] / nv;
        r.z += m.xyz[3 * v + 2] / nv;
    }
    return r;
}

}  // namespace

int build_graph(const HostMesh &m, const ep_graph_desc *d, const ep_graph_params *p, const ep_params *jp,
                GraphPlan *g, std::string *err) {
    const int64_t n = d->n_nodes, ne = d->n_edges, nj = d->n_junctions;
    if (n < 0 || ne < 0 || nj < 0 || (n > 0 && !d->xyz) || (ne > 0 && !d->edges) ||
        (nj > 0 && (!d->junction_node || !d->junction_cell))) {
        *err = "graph: negative size or NULL array";
        return EP_EINVAL;
    }
    if (n >= (int64_t(1) << 31) || ne >= (int64_t(1) << 30)) {
        *err = "graph: too many nodes or edges";
        return EP_EINVAL;
    }
    if (!(p->D >= 0.0) || !(p->radius >= 0.0) || !(p->duration >= 0.0) || !(p->delay_ortho >= 0.0) ||
        !(p->delay_anti >= 0.0) || p->default_mode < EP_PMJ_RESISTIVE || p->default_mode > EP_PMJ_CELL) {
        *err = "graph: bad coupling parameters";
        return EP_EINVAL;
    }
    std::vector<uint8_t> model(n, EP_STEWART), pset(n, 0), smask(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (d->node_model) model[i] = d->node_model[i];
        if (d->node_param_set) pset[i] = d->node_param_set[i];
        if (d->node_stim_mask) smask[i] = d->node_stim_mask[i];
        if (model[i] >= EP_N_MODELS || pset[i] >= jp->n_sets) {
            *err = "graph: node " + std::to_string(i) + " has an unknown model or parameter set";
            return EP_EINVAL;
        }
    }
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t a = d->edges[2 * e], b = d->edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) {
            *err = "graph: bad edge " + std::to_string(e);
            return EP_EINVAL;
        }
        if (d->edge_D && !(d->edge_D[e] >= 0.0)) {
            *err = "graph: negative edge diffusivity";
            return EP_EINVAL;
        }
    }
    // node order: grouped by model, input order inside a group
    g->n = n;
    g->new2old.resize(n);
    std::vector<int32_t> old2new(n);
    for (int md = 0; md <= EP_N_MODELS; ++md) g->model_off[md] = 0;
    for (int64_t i = 0; i < n; ++i) g->model_off[model[i] + 1]++;
    for (int md = 0; md < EP_N_MODELS; ++md) g->model_off[md + 1] += g->model_off[md];
    {
        int64_t fill[EP_N_MODELS];
        for (int md = 0; md < EP_N_MODELS; ++md) fill[md] = g->model_off[md];
        for (int64_t i = 0; i < n; ++i) {
            const int64_t k = fill[model[i]]++;
            g->new2old[k] = int32_t(i);
            old2new[i] = int32_t(k);
        }
    }
    g->pset.resize(n);
    g->smask.resize(n);
    for (int64_t k = 0; k < n; ++k) {
        g->pset[k] = pset[g->new2old[k]];
        g->smask[k] = smask[g->new2old[k]];
    }
    // vertex-based FV coefficients and the subcycle count
    std::vector<std::vector<std::pair<int32_t, double>>> adj(n);   // (neighbour, D / L)
    std::vector<double> sumL(n, 0.0);
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t a = d->edges[2 * e], b = d->edges[2 * e + 1];
        const double *xa = d->xyz + 3 * int64_t(a), *xb = d->xyz + 3 * int64_t(b);
        const double L = std::sqrt((xa[0] - xb[0]) * (xa[0] - xb[0]) + (xa[1] - xb[1]) * (xa[1] - xb[1]) +
                                   (xa[2] - xb[2]) * (xa[2] - xb[2]));
        if (!(L > 0.0)) {
            *err = "graph: edge " + std::to_string(e) + " has zero length";
            return EP_EINVAL;
        }
        const double D = d->edge_D ? d->edge_D[e] : p->D;
        adj[old2new[a]].push_back({old2new[b], D / L});
        adj[old2new[b]].push_back({old2new[a], D / L});
        sumL[old2new[a]] += L;
        sumL[old2new[b]] += L;
    }
    g->row.assign(n + 1, 0);
    g->col.clear();
    g->coef.clear();
    double rho = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        std::sort(adj[i].begin(), adj[i].end());
        double rowsum = 0.0;
        for (auto &pr : adj[i]) {
            const double c = 2.0 * pr.second / sumL[i];
            g->col.push_back(pr.first);
            g->coef.push_back(c);
            rowsum += c;
        }
        g->row[i + 1] = int32_t(g->col.size());
        rho = std::max(rho, 2.0 * rowsum);
    }
    g->rho = rho;
    g->substeps = std::max(1, int(std::ceil(jp->dt * rho / 1.8)));
    // junctions
    std::vector<int32_t> cell_old2new(m.n_cells);
    for (int64_t c = 0; c < m.n_cells; ++c) cell_old2new[m.cell_new2old[c]] = int32_t(c);
    g->jnode.resize(nj);
    g->jcell.resize(nj);
    g->jmode.resize(nj);
    for (int64_t j = 0; j < nj; ++j) {
        const int32_t a = d->junction_node[j], c = d->junction_cell[j];
        const uint8_t mode = d->junction_mode ? d->junction_mode[j] : uint8_t(p->default_mode);
        const bool cellsrc = mode == EP_PMJ_CELL;   // the source is a cell, not a graph node
        if (a < 0 || a >= (cellsrc ? m.n_cells : n) || c < 0 || c >= m.n_cells || mode > EP_PMJ_CELL) {
            *err = "graph: bad junction " + std::to_string(j);
            return EP_EINVAL;
        }
        g->jnode[j] = cellsrc ? cell_old2new[a] : old2new[a];
        g->jcell[j] = cell_old2new[c];
        g->jmode[j] = mode;
    }
    // junctions at each graph node (cell-to-cell nodes have no graph side)
    g->node_junc_ptr.assign(n + 1, 0);
    for (int64_t j = 0; j < nj; ++j)
        if (g->jmode[j] != EP_PMJ_CELL) g->node_junc_ptr[g->jnode[j] + 1]++;
    for (int64_t i = 0; i < n; ++i) g->node_junc_ptr[i + 1] += g->node_junc_ptr[i];
    g->node_junc.resize(std::max<int64_t>(g->node_junc_ptr[n], 0));
    {
        std::vector<int32_t> fill(g->node_junc_ptr.begin(), g->node_junc_ptr.end() - 1);
        for (int64_t j = 0; j < nj; ++j)
            if (g->jmode[j] != EP_PMJ_CELL) g->node_junc[fill[g->jnode[j]]++] = int32_t(j);
    }
    // cell-side entries: the junction cell of resistive junctions, every cell within
    // `radius` of the junction cell for triggered ones (spatial hash of centroids)
    std::vector<std::pair<int32_t, int32_t>> ent;
    bool any_trig = false;
    for (int64_t j = 0; j < nj; ++j) {
        if (g->jmode[j] == EP_PMJ_RESISTIVE) ent.push_back({g->jcell[j], int32_t(j)});
        else any_trig = true;
        // the source cell of a cell-to-cell node: records its crossings, and is excited back (two-way)
        if (g->jmode[j] == EP_PMJ_CELL) ent.push_back({g->jnode[j], int32_t(j) | kJunctionSource});
    }
    if (any_trig) {
        const double r = p->radius;
        if (r > 0.0) {
            const double cs = r;
            std::unordered_map<uint64_t, std::vector<int32_t>> grid;
            auto key = [](int64_t a, int64_t b, int64_t c) {
                return (uint64_t(a + (1 << 20)) << 42) | (uint64_t(b + (1 << 20)) << 21) | uint64_t(c + (1 << 20));
            };
            std::vector<P3> cen(m.n_cells);
            for (int64_t c = 0; c < m.n_cells; ++c) {
                cen[c] = centroid(m, c);
                grid[key(int64_t(std::floor(cen[c].x / cs)), int64_t(std::floor(cen[c].y / cs)),
                         int64_t(std::floor(cen[c].z / cs)))]
                    .push_back(int32_t(c));
            }
            for (int64_t j = 0; j < nj; ++j) {
                if (g->jmode[j] == EP_PMJ_RESISTIVE) continue;
                const P3 x0 = cen[g->jcell[j]];
                const uint8_t medium = m.kind.empty() ? 0 : m.kind[g->jcell[j]];
                const int64_t bx = int64_t(std::floor(x0.x / cs)), by = int64_t(std::floor(x0.y / cs)),
                              bz = int64_t(std::floor(x0.z / cs));
                for (int64_t dx = -1; dx <= 1; ++dx)
                    for (int64_t dy = -1; dy <= 1; ++dy)
                        for (int64_t dz = -1; dz <= 1; ++dz) {
                            auto it = grid.find(key(bx + dx, by + dy, bz + dz));
                            if (it == grid.end()) continue;
                            for (int32_t c : it->second) {
                                if ((m.kind.empty() ? 0 : m.kind[c]) != medium) continue;   // the target's medium
                                const double ex = cen[c].x - x0.x, ey = cen[c].y - x0.y, ez = cen[c].z - x0.z;
                                if (c == g->jcell[j] || std::sqrt(ex * ex + ey * ey + ez * ez) <= r)
                                    ent.push_back({c, int32_t(j)});
                            }
                        }
            }
        } else {
            for (int64_t j = 0; j < nj; ++j)
                if (g->jmode[j] != EP_PMJ_RESISTIVE) ent.push_back({g->jcell[j], int32_t(j)});
        }
    }
    std::sort(ent.begin(), ent.end());
    g->tgt_cell.resize(ent.size());
    g->tgt_junc.resize(ent.size());
    for (size_t k = 0; k < ent.size(); ++k) {
        g->tgt_cell[k] = ent[k].first;
        g->tgt_junc[k] = ent[k].second;
    }
    g->p = *p;
    return EP_OK;
}

}  // namespace ep
