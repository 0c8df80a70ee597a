// Host-side multigrid hierarchy (see mg_host.cpp).
#pragma once

#include <vector>

#include "rte_internal.h"

namespace rte {

struct MGHostLevel {
    int m = 0;                       // m x m squares on this level
    Stencil st;                      // 7-point pattern
    std::vector<double> vals;        // [slots][nnz][bs][bs]
    // transfer to the next coarser level (empty on the coarsest)
    std::vector<int> p0, p1;         // prolongation: coarse nodes per fine node
    std::vector<float> w0, w1;       //   and their weights (p1 = -1: one node)
    std::vector<int> rptr, ridx;     // restriction P^T: CSR over coarse nodes
    std::vector<float> rw;
};

struct MGHost {
    std::vector<MGHostLevel> levels;
    int bs = 1, slots = 1;
    int coarse_nodes = 0;
    bool dense_coarse = false;       // coarsest level solved by a dense inverse
};

Stencil stencil_of_square(int m);

// Builds levels m, m/2, ... from the fine pattern and values until the mesh
// no longer halves or has at most 25 nodes.
int build_hierarchy(int m, const Stencil& fine, const std::vector<double>& vals0, int slots,
                    int bs, int max_coarse_nodes, MGHost& out);

// Inverse of sum_s weights[s] vals[s] on level L (dense, (n bs)^2 floats).
int coarse_dense_inverse(const MGHostLevel& L, const std::vector<double>& weights, int slots,
                         int bs, std::vector<float>& inv);

// Inverses of the diagonal bs x bs blocks (slot 0) of level L.
int block_diag_inverse(const MGHostLevel& L, int bs, std::vector<float>& dinv);

}  // namespace rte
