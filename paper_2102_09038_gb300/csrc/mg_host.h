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

// Builds levels m, floor(m/2), ... from the fine pattern and values while
// the level has m >= 4 and more than max_coarse_nodes nodes; the coarsest is
// marked for a dense inverse when it has at most max_coarse_nodes nodes.
int build_hierarchy(int m, const Stencil& fine, const std::vector<double>& vals0, int slots,
                    int bs, int max_coarse_nodes, MGHost& out);

// Dense matrix sum_s weights[s] vals[s] on level L ((n bs)^2 doubles,
// row-major); weights empty means all ones.
void coarse_dense_matrix(const MGHostLevel& L, const std::vector<double>& weights, int slots,
                         int bs, std::vector<double>& A);

// Inverses of the diagonal bs x bs blocks (slot 0) of level L.
int block_diag_inverse(const MGHostLevel& L, int bs, std::vector<float>& dinv);

// The 7 stencil directions of the "/"-mesh: self, +x, -x, +y, -y, +x+y, -x-y.
// ELL form of slot values on a level: out[s][dir][node][bs][bs] (zero where
// the neighbour does not exist).  Fails if an entry is not one of the 7.
int to_ell(const MGHostLevel& L, int slots, int bs, std::vector<double>& out);

}  // namespace rte
