// Host planning of a conduction graph attached to a job: node ordering by
// cell model, the vertex-based FV coefficients (Sec. 3.2), the subcycle
// count, and the junction tables on both sides (Sec. 3.3).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ep.h"
#include "planner.h"

namespace ep {

struct GraphPlan {
    int64_t n = 0;
    std::vector<int32_t> new2old;            // internal node -> caller node
    std::vector<uint8_t> pset, smask;        // internal order
    int64_t model_off[EP_N_MODELS + 1] = {0, 0, 0, 0};
    std::vector<int32_t> row, col;           // CSR of neighbours (internal numbering)
    std::vector<double> coef;                // c_ij = 2 D_ij / (L_ij sum_k L_ik)
    int substeps = 1;
    double rho = 0.0;                        // bound of the graph operator's spectral radius
    std::vector<int32_t> jnode, jcell;       // internal graph node / internal cell
    std::vector<uint8_t> jmode;
    std::vector<int32_t> node_junc_ptr, node_junc;   // junctions of each node
    std::vector<int32_t> tgt_cell, tgt_junc;         // (cell, junction) entries, sorted by cell
    ep_graph_params p{};
};

// Validate and plan a graph for mesh m and job parameters jp (dt, number of
// parameter sets). Returns EP_OK or an error code with a message.
int build_graph(const HostMesh &m, const ep_graph_desc *d, const ep_graph_params *p, const ep_params *jp,
                GraphPlan *g, std::string *err);

}  // namespace ep
