// Internal declarations shared by the translation units of librte.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rte.h"

namespace rte {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define RTE_CUDA_TRY(expr)                                                   \
    do {                                                                     \
        cudaError_t e__ = (expr);                                            \
        if (e__ != cudaSuccess)                                              \
            return ::rte::fail(RTE_ERR_CUDA, std::string(#expr) + ": " +     \
                                                 cudaGetErrorString(e__));   \
    } while (0)

#define RTE_TRY(expr)                                                        \
    do {                                                                     \
        int rc__ = (expr);                                                   \
        if (rc__ != RTE_OK) return rc__;                                     \
    } while (0)

// ---------------------------------------------------------- host meshes
// Uniform "/"-triangulation of the unit square (Section 4, T_h^R).
struct SquareMesh {
    int m = 0, n_nodes = 0, n_cells = 0;
    std::vector<int> cell_nodes;     // 3 per cell, counter-clockwise
    std::vector<double> area;        // per cell
    std::vector<double> grad;        // 6 per cell: dphi_a/dx (a=0..2), dphi_a/dy
};
SquareMesh make_square(int m);

// Octahedron refined `levels` times (Section 6); only the representatives of
// the antipodal pairs (children of the four upper faces) are kept.
struct SphereMesh {
    int levels = 0, n = 0;
    std::vector<double> verts;       // 3 per vertex (unit vectors)
    std::vector<int> tri;            // 3 vertex ids per representative
};
SphereMesh make_sphere(int levels);
// Level-r rule on one spherical triangle (refine r times, one node per
// sub-triangle at its normalised vertex mean, weight its exact area); appends
// 4^r points (3 doubles each) and weights at index `count`.
void quad_one(const double* a, const double* b, const double* c, int r, double* pts, double* w,
              int& count);
bool inv3(const double* A, double* Ai);
// Pairs (k, k') where K_k' or -K_k' shares a vertex with K_k (sorted per k).
void sphere_near_pairs(const SphereMesh& S, std::vector<int>& ptr, std::vector<int>& idx);

// Sparse 7-point node stencil (row = node, sorted columns, diagonal index).
struct Stencil {
    std::vector<int> ptr, col, diag;
};

// ------------------------------------------------------------ host setup
// Everything the device needs, assembled on the host.
struct HostSystem {
    int m, levels, nRp, nRm, nSp, nSm, dP, dM;
    double g, c, gamma;
    SquareMesh mesh;
    SphereMesh sphere;
    Stencil st;
    // stencil values, kVal* slots of nnz doubles each
    std::vector<double> sval;
    std::vector<int> adj_ptr, adj_cell, adj_loc;   // node -> (cell, vertex)
    std::vector<double> cell_D;                    // 6 per cell (D1[a], D2[a])
    std::vector<double> cell_at, cell_as;          // |T| sigma_t, |T| sigma_s
    // angular
    std::vector<double> m_, omx, omy, A1, A2, MSm, MSm_inv, e0s;
    std::vector<double> quad_near_pts, quad_near_w;   // per triangle
    std::vector<double> quad_far_pts, quad_far_w;
    std::vector<double> quad_near_psi, quad_far_psi;  // psi_i at the nodes
    std::vector<int> near_ptr, near_idx;               // vertex-sharing pairs
};

enum StencilSlot {
    kMt = 0,    // sigma_t-weighted P1 mass M_t^+
    kMs = 1,    // sigma_s-weighted P1 mass M_s^+
    kMu = 2,    // unit P1 mass (source)
    kBx = 3,    // P1 boundary mass on x = 0 and x = 1
    kBy = 4,    // P1 boundary mass on y = 0 and y = 1
    kK11 = 5,   // D_1^T (M_t^-)^{-1} D_1
    kK12 = 6,   // D_1^T (M_t^-)^{-1} D_2 + D_2^T (M_t^-)^{-1} D_1
    kK22 = 7,   // D_2^T (M_t^-)^{-1} D_2
    kSlots = 8
};

int build_host_system(const rte_problem& p, const rte_options& o,
                      HostSystem& hs);

constexpr int kRFar = 2;
constexpr int kRNear = 4;

}  // namespace rte
