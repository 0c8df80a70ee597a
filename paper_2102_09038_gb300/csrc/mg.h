// Device-side multigrid hierarchy shared by the E_0 and E_c solvers.
//
// Every level is the uniform (m+1) x (m+1) node grid of an m x m "/"-mesh;
// level l+1 is the floor(m/2)-mesh of level l.
// Operators are stored in ELL form over the 7 stencil directions
//   0: self, 1: +x, 2: -x, 3: +y, 4: -y, 5: +x+y, 6: -x-y
// (zero coefficients where a neighbour does not exist), so neighbour,
// restriction and prolongation indices are computed, not looked up.
#pragma once

namespace rte {

constexpr int kMaxMGLevels = 14;
// a coarsest level of at most this many nodes is solved by dense inverses
constexpr int kDenseCoarseNodes = 300;

struct MGDeviceLevel {
    int m = 0, n = 0;
    const float* val = nullptr;    // E_c: [7][n][d][d], blocks transposed
    const float* dinv = nullptr;   // E_c: [n][d][d] inverse diagonal blocks, transposed
    const float* sv = nullptr;     // E_0: six spatial parts [n][7][8]; E_c: Q terms [n][7][Qp]
    float *X = nullptr, *Xt = nullptr, *B = nullptr;   // work vectors
    // restriction from the next finer level: for each node of this level,
    // rwid fine nodes and weights (zero-weight padding); unset on level 0
    const int* ridx = nullptr;
    const float* rw = nullptr;
    int rwid = 0;
};

struct MGDevice {
    int L = 0, nu = 2, cap_cols = 0;
    bool dense = false;
    const float* cinv = nullptr;   // coarsest dense inverse(s)
    int Q = 0;                     // E_c only: number of Kronecker terms (0: blocks)
    const float* G = nullptr;      // E_c only: angular blocks of the terms [Q][d][d]
    const float* w8 = nullptr;     // E_0 only: per-direction weights [nSp][8], six used
    const float* wq = nullptr;     // E_0 only: the same weights [6][nSp]
    MGDeviceLevel lev[kMaxMGLevels];
    const MGDeviceLevel* dev_lev = nullptr;   // copy of lev[0 .. L) in device memory
};

}  // namespace rte
