// Host planner: mesh ingest, reverse Cuthill-McKee renumbering, face
// matching and the FP64 folding of the finite-volume stencil (Sec. 3.2,
// Eqs. 2-3, 7-8) into per-cell coefficients for the device step.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ep.h"

namespace ep {

struct HostMesh {
    int64_t n_nodes = 0, n_cells = 0;
    std::vector<double> xyz;          // [3 n_nodes], internal node order
    std::vector<int32_t> tet;         // [4 n_cells], internal cell order, positive orientation; a triangle
                                      // (kind 1) holds its 3 nodes and repeats the first in slot 3
    std::vector<uint8_t> kind;        // [n_cells] 0 tetrahedron, 1 shell triangle (face k = edge opposite node k)
    std::vector<int32_t> nbr;         // [4 n_cells] cell across the face opposite vertex k, -1 boundary
    std::vector<int32_t> opp;         // [4 n_cells] neighbour's vertex off that face, -1 boundary
    std::vector<uint8_t> model, pset, smask;
    std::vector<double> fibre;        // [3 n_cells] or empty (isotropic)
    std::vector<int32_t> cell_new2old, node_new2old;
    int64_t model_off[EP_N_MODELS + 1] = {0, 0, 0, 0};
    int64_t n_interior_faces = 0;
    std::vector<int64_t> n2c_ptr;     // node -> incident cells (internal numbering, sorted)
    std::vector<int32_t> n2c;
    int index_width = 0;              // ep_mesh_desc::index_width (0 automatic, 16, 32)
};

// Validate, orient, match faces, renumber (RCM, grouped by model).
int build_mesh(const ep_mesh_desc *d, HostMesh *m, std::string *err);

// FP64 folded coefficients of one job. For cell c, the diffusion term is
//   sum_k wa[4c+k] vn[tet[4c+k]] + sum_k wb[4c+k] vn[opp[4c+k]]
//   + sum_k q[4c+k] (V[nbr[4c+k]] - V[c]),
// vn the inverse-distance node values, vn[n] = sum_j nw[j] V[n2c[j]].
struct Coeffs {
    std::vector<double> wa, wb, q;    // [4 n_cells]
    std::vector<double> nw;           // aligned with HostMesh::n2c
    double gershgorin = 0.0;          // max row sum of |operator|
};
int build_coeffs(const HostMesh &m, const ep_params *p, Coeffs *c, std::string *err);

// Spectral radius estimate of the folded operator by power iteration.
double power_radius(const HostMesh &m, const Coeffs &c, int iters);

// Device index layout of a job's step: the sliced-ELL node -> cell table
// (slices of 32 nodes, column-major inside a slice; src[e] indexes
// HostMesh::n2c and Coeffs::nw, -1 = pad) and the cells' gather indices
// (own vertices, the vertex of the neighbour opposite each face, the
// neighbour across each face; on a boundary face the cell's own vertex 0 and
// the cell itself). Indices are stored either as 32-bit values or, where the
// numbering allows, as 16-bit offsets -- the cells' gather indices (idx16)
// and the ELL entries (col16) independently:
//   - a cell's 8 node indices relative to nbase[c >> 8] (unsigned; the base is
//     the smallest node index of the 256-cell run);
//   - a cell's 4 neighbours relative to the cell itself (signed);
//   - the ELL entries of a slice relative to cbase[slice] (unsigned). The
//     cells around one node span several RCM levels (about six times the
//     neighbour bandwidth), so this form fits smaller meshes only.
struct Sell {
    std::vector<int64_t> slice_ptr;   // [n_slices + 1] entry offsets
    std::vector<int32_t> col;         // cell index per entry (pads repeat a valid cell)
    std::vector<int64_t> src;
    bool idx16 = false, col16ok = false;
    std::vector<uint16_t> col16;      // [entries] ELL offsets from cbase
    std::vector<int32_t> cbase;       // [n_slices]
    std::vector<uint16_t> cidx16;     // [8 n_cells] na then nb offsets from nbase
    std::vector<int16_t> nbr16;       // [4 n_cells] neighbour offsets from the cell
    std::vector<int32_t> nbase;       // [(n_cells + 255) / 256]
};
void build_sell(const HostMesh &m, Sell *s);

// The 32-bit gather indices of cell c: own vertices, opposite vertices,
// neighbours (boundary faces: own vertex 0 and the cell itself).
void cell_gather_indices(const HostMesh &m, int64_t c, int32_t na[4], int32_t nb[4], int32_t nc[4]);

}  // namespace ep
