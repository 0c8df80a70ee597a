// H^2 compression of S^+ and S^- (Section 5.2): host-side plan shared by
// h2_build.cpp (cluster tree, boxes, block tree, block lists) and h2.cu
// (device set-up of the matrices and the block-sparse apply).
#pragma once

#include <vector>

namespace rte {

constexpr int kH2B = 64;      // width of the blocks of every block-sparse product
constexpr int kH2Leaf = 64;   // representatives per leaf cluster (n_min)

// One block-sparse product Out[:, 64 out_blk[j] ..] (+)= sum over the entries
// e of row j of In[:, 64 in_blk[e] ..] * B_e, B_e a 64 x 64 matrix (mat[e]:
// index into the matrix pool, or for the coupling stage the sign of the part).
struct H2List {
    std::vector<int> out_blk, ptr, in_blk, mat;
};

struct H2Plan {
    int levels = 0, n = 0, p = 0, k = 0;
    int ld = 0;     // leaf depth
    int dmin = 0;   // shallowest depth holding a far block (ld when none)
    double eta = 0;
    std::vector<int> depth_off;   // cluster id of (d, 0), d = dmin..ld
    int ncl = 0;                  // clusters with a basis (depths dmin..ld)
    std::vector<double> lo, hi;   // boxes of those clusters [ncl][3]
    std::vector<double> xi;       // normalised tensor points [ncl][64][3] (zero padded)
    std::vector<double> nodes;    // per-axis Chebyshev nodes [ncl][p][3]
    struct Blk { int depth, t, c, sign; };
    std::vector<Blk> far, near;
    // near blocks with the two parts merged: leaf pair (t, c), flags bit 0
    // direct part near, bit 1 mirror part near
    struct NearPair { int t, c, flags; };
    std::vector<NearPair> nearm;
    int leaves() const { return 4 << (2 * ld); }
    int count(int d) const { return 4 << (2 * d); }
    int id(int d, int t) const { return depth_off[d - dmin] + t; }
};

// Cluster tree, boxes (from the far-rule points [n][qf][3]), Chebyshev
// nodes and block tree.  Returns false for a degenerate box.
bool h2_plan(int levels, double eta, int p, const std::vector<double>& far_pts, int qf,
             H2Plan& plan);

// Matrix-pool layout of one parity (m = 1 for S^+, 3 for S^-): leaf bases
// (leaves * m), transfer matrices (clusters below dmin), near blocks
// (near pairs * m * m).
struct H2Pool {
    int m = 1;
    long long leaf0 = 0, transfer0 = 0, near0 = 0, total = 0;
    long long leaf(int t, int chunk) const { return leaf0 + (long long)t * m + chunk; }
    long long transfer(const H2Plan& P, int d, int c) const {
        return transfer0 + P.id(d, c) - P.count(P.dmin);
    }
    long long nearb(int pair, int a, int b) const { return near0 + ((long long)pair * m + a) * m + b; }
};
H2Pool h2_pool(const H2Plan& P, int m);

// Block lists of the apply stages for one parity:
// up_leaf (X -> Xh leaves), up[d] (Xh depth d+1 -> depth d, d = ld-1..dmin),
// couple (Xh -> Yh, all depths), down[d] (Yh depth d -> depth d+1,
// d = dmin..ld-1, transposed transfers), down_leaf (Yh leaves -> Y,
// transposed bases), near (X -> Y, accumulated).
struct H2Lists {
    H2List up_leaf, couple, down_leaf, near;
    std::vector<H2List> up, down;   // indexed by d - dmin
};
void h2_lists(const H2Plan& P, const H2Pool& pool, H2Lists& L);

// Limit of one mbarrier wait of the tensor-core H^2 products (SM cycles).
int h2_set_wait_cycles(long long cycles);

}  // namespace rte
