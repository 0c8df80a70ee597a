// Device-side multigrid hierarchy shared by the E_0 and E_c solvers.
#pragma once

namespace rte {

constexpr int kMaxMGLevels = 14;

struct MGDeviceLevel {
    int n = 0, nnz = 0;
    const int *ptr = nullptr, *col = nullptr, *diag = nullptr;
    const float* val = nullptr;    // E_0: [6][nnz]; E_c: [nnz][d][d]
    const float* dinv = nullptr;   // E_c: [n][d][d] inverse diagonal blocks
    const int *rptr = nullptr, *ridx = nullptr, *p0 = nullptr, *p1 = nullptr;
    const float *rw = nullptr, *w0 = nullptr, *w1 = nullptr;
    float *X = nullptr, *Xt = nullptr, *B = nullptr;   // work vectors
};

struct MGDevice {
    int L = 0, nu = 2, cap_cols = 0;
    bool dense = false;
    const float* cinv = nullptr;   // coarsest dense inverse(s)
    const float* e0s = nullptr;    // E_0 only: per-direction weights [nSp][6]
    MGDeviceLevel lev[kMaxMGLevels];
};

}  // namespace rte
