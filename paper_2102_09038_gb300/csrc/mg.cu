// Multigrid-preconditioned conjugate gradients, each solve in one persistent
// cooperative kernel:
//  * E_0^{-1} (eq. equivalence_bE_bE0): the n_S^+ decoupled direction blocks,
//    block k = gamma (a11 K11 + a12 K12 + a22 K22) + om^x B_x + om^y B_y +
//    m_k M_t^+, all (rhs, direction) columns at once, each column stopping
//    on its own relative residual.  This is the "multigrid" route the paper
//    names for these anisotropic diffusion blocks (Section 5.5).
//  * E_c^{-1} (Section 5.4): the coarse Galerkin system, d x d blocks on the
//    node stencil, one CG per right-hand side.
// The preconditioner is one symmetric V-cycle in FP32 on the nested meshes
// (damped Jacobi / block Jacobi smoothing, nu sweeps before and after,
// restriction P^T, dense inverse on the coarsest level); the CG recurrences
// run in the solve's precision T with FP64 reductions.  Blocks meet at
// bounded grid barriers (persist.cuh).
#include <cuda_runtime.h>

#include <algorithm>

#include "device.h"
#include "mg.h"
#include "persist.cuh"
#include "rte_internal.h"

namespace rte {

namespace {

constexpr float kOmega = 0.7f;          // Jacobi damping
constexpr int kCoarseSweeps = 30;       // coarsest-level sweeps without a dense inverse

// ================================================================ E_0 V-cycle
struct E0Level {
    int n;
    const int *ptr, *col, *diag;
    const float* val;      // [6][nnz] in the order of e0s
    int nnz;
    const int *rptr, *ridx, *p0, *p1;
    const float *rw, *w0, *w1;
    float *X, *Xt, *B;     // [n][ncols]
};

__device__ __forceinline__ void e0_load_s(const float* e0s, int k, float* s) {
#pragma unroll
    for (int q = 0; q < 6; ++q) s[q] = __ldg(e0s + 6 * k + q);
}

__device__ __forceinline__ float e0_c(const E0Level& L, const float* s, int p) {
    const float* v = L.val + p;
    return s[0] * __ldg(v) + s[1] * __ldg(v + L.nnz) + s[2] * __ldg(v + 2 * L.nnz) +
           s[3] * __ldg(v + 3 * L.nnz) + s[4] * __ldg(v + 4 * L.nnz) +
           s[5] * __ldg(v + 5 * L.nnz);
}

// y = A x at item (i, c), and the diagonal coefficient
__device__ __forceinline__ float e0_apply(const E0Level& L, const float* s, const float* x,
                                          int i, int c, int ncols, float& dg) {
    float y = 0.f;
    for (int p = L.ptr[i]; p < L.ptr[i + 1]; ++p)
        y += e0_c(L, s, p) * ldg2(x + (size_t)L.col[p] * ncols + c);
    dg = e0_c(L, s, L.diag[i]);
    return y;
}

struct E0MG {
    int L, ncols, nSp, nu;
    bool dense;
    const float* cinv;     // [nSp][n_c][n_c]
    const float* e0s;      // [nSp][6]
    E0Level lev[kMaxMGLevels];
};

#define GSTRIDE(e, total)                                                        \
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (total); \
         e += (size_t)gridDim.x * blockDim.x)

// One symmetric V-cycle on B_0; returns the buffer holding z on level 0.
__device__ bool e0_vcycle(const E0MG& mg, GridBar* bar, float*& z) {
    const int nc = mg.ncols;
    int cur[kMaxMGLevels];
    for (int l = 0; l < mg.L; ++l) cur[l] = 0;
    auto buf = [&](int l, int which) { return which ? mg.lev[l].Xt : mg.lev[l].X; };
    // ---- pre-smoothing from zero, residual, restriction
    auto jacobi = [&](int l) -> bool {
        const E0Level& Lv = mg.lev[l];
        const float* x = buf(l, cur[l]);
        float* xt = buf(l, cur[l] ^ 1);
        GSTRIDE(e, (size_t)Lv.n * nc) {
            const int i = (int)(e / nc), c = (int)(e % nc);
            float s[6];
            e0_load_s(mg.e0s, c % mg.nSp, s);
            float dg;
            const float y = e0_apply(Lv, s, x, i, c, nc, dg);
            xt[e] = ldg2(x + e) + kOmega * (ldg2(Lv.B + e) - y) / dg;
        }
        cur[l] ^= 1;
        return grid_sync(bar);
    };
    auto first = [&](int l) -> bool {
        const E0Level& Lv = mg.lev[l];
        float* x = buf(l, 0);
        GSTRIDE(e, (size_t)Lv.n * nc) {
            const int i = (int)(e / nc), c = (int)(e % nc);
            float s[6];
            e0_load_s(mg.e0s, c % mg.nSp, s);
            x[e] = kOmega * ldg2(Lv.B + e) / e0_c(Lv, s, Lv.diag[i]);
        }
        cur[l] = 0;
        return grid_sync(bar);
    };
    for (int l = 0; l + 1 < mg.L; ++l) {
        const E0Level& Lv = mg.lev[l];
        if (!first(l)) return false;
        for (int k = 1; k < mg.nu; ++k)
            if (!jacobi(l)) return false;
        // residual into the spare buffer
        const float* x = buf(l, cur[l]);
        float* t = buf(l, cur[l] ^ 1);
        GSTRIDE(e, (size_t)Lv.n * nc) {
            const int i = (int)(e / nc), c = (int)(e % nc);
            float s[6];
            e0_load_s(mg.e0s, c % mg.nSp, s);
            float dg;
            t[e] = ldg2(Lv.B + e) - e0_apply(Lv, s, x, i, c, nc, dg);
        }
        if (!grid_sync(bar)) return false;
        const E0Level& Cv = mg.lev[l + 1];
        GSTRIDE(e, (size_t)Cv.n * nc) {
            const int I = (int)(e / nc), c = (int)(e % nc);
            float acc = 0.f;
            for (int q = Lv.rptr[I]; q < Lv.rptr[I + 1]; ++q)
                acc += Lv.rw[q] * ldg2(t + (size_t)Lv.ridx[q] * nc + c);
            Cv.B[e] = acc;
        }
        if (!grid_sync(bar)) return false;
    }
    // ---- coarsest level
    {
        const int l = mg.L - 1;
        const E0Level& Lv = mg.lev[l];
        if (mg.dense) {
            float* x = buf(l, 0);
            GSTRIDE(e, (size_t)Lv.n * nc) {
                const int i = (int)(e / nc), c = (int)(e % nc);
                const float* row = mg.cinv + ((size_t)(c % mg.nSp) * Lv.n + i) * Lv.n;
                float acc = 0.f;
                for (int j = 0; j < Lv.n; ++j) acc += __ldg(row + j) * ldg2(Lv.B + (size_t)j * nc + c);
                x[e] = acc;
            }
            cur[l] = 0;
            if (!grid_sync(bar)) return false;
        } else {
            if (!first(l)) return false;
            for (int k = 1; k < kCoarseSweeps; ++k)
                if (!jacobi(l)) return false;
        }
    }
    // ---- prolongation and post-smoothing
    for (int l = mg.L - 2; l >= 0; --l) {
        const E0Level& Lv = mg.lev[l];
        float* x = buf(l, cur[l]);
        const float* xc = buf(l + 1, cur[l + 1]);
        GSTRIDE(e, (size_t)Lv.n * nc) {
            const int i = (int)(e / nc), c = (int)(e % nc);
            float v = Lv.w0[i] * ldg2(xc + (size_t)Lv.p0[i] * nc + c);
            if (Lv.p1[i] >= 0) v += Lv.w1[i] * ldg2(xc + (size_t)Lv.p1[i] * nc + c);
            x[e] = ldg2(x + e) + v;
        }
        if (!grid_sync(bar)) return false;
        for (int k = 0; k < mg.nu; ++k)
            if (!jacobi(l)) return false;
    }
    z = buf(0, cur[0]);
    return true;
}

// ================================================================ E_0 PCG
template <typename T>
struct E0Args {
    int nRp, nSp, nrhs, ncols, kTiles, chunks, units, maxit;
    double tol2;
    const int* st_ptr;
    const int* st_col;
    const T* coef;      // level-0 coefficients [nnz][nSp] in the CG precision
    const double* B;
    double* X;
    T* R;
    T* P;
    T* AP;
    double* acc;        // [3 slots][3][ncols]: pAp, rz, rr
    double* bb;
    GridBar* bar;
    SolveStatus* status;
    E0MG mg;
};

constexpr int kChunk = 64;   // nodes per work unit (8 rows x 8 passes)

template <typename T>
__device__ __forceinline__ double* slot(const E0Args<T>& a, int s, int q) {
    return a.acc + ((size_t)s * 3 + q) * a.ncols;
}

__device__ void col_add(double v, double* sh, double* dst, int col, bool valid) {
    const int kx = threadIdx.x & 31, ny = threadIdx.x >> 5;
    sh[ny * 32 + kx] = v;
    __syncthreads();
    if (ny == 0) {
        double s = 0.0;
        for (int y = 0; y < 8; ++y) s += sh[y * 32 + kx];
        if (valid) atomicAdd(dst + col, s);
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_e0_pcg(E0Args<T> a) {
    __shared__ double sh[256];
    __shared__ int s_stop;
    const int kx = threadIdx.x & 31, ny = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_stop = 0;
    const int nc = a.ncols;
    float* B0 = a.mg.lev[0].B;
    // unit u -> (rhs r, direction tile kt, node chunk)
#define UNIT_LOOP                                                   \
    for (int u = blockIdx.x; u < a.units; u += gridDim.x) {         \
        const int chunk = u % a.chunks;                             \
        const int kt = (u / a.chunks) % a.kTiles;                   \
        const int r = u / (a.chunks * a.kTiles);                    \
        const int k = kt * 32 + kx;                                 \
        const bool kv = k < a.nSp;                                  \
        const int col = r * a.nSp + k;
#define UNIT_END }
#define NODE_LOOP                                                   \
    for (int t = 0; t < kChunk / 8; ++t) {                          \
        const int i = chunk * kChunk + ny + 8 * t;                  \
        if (i >= a.nRp) continue;                                   \
        const size_t e = ((size_t)r * a.nRp + i) * a.nSp + k;       \
        const size_t em = (size_t)i * nc + col;
    // ------------------------------------------------------------ init
    UNIT_LOOP
        double pbb = 0.0;
        if (kv) {
            NODE_LOOP
                const T b = static_cast<T>(a.B[e]);
                a.X[e] = 0.0;
                a.R[e] = b;
                B0[em] = static_cast<float>(b);
                pbb += (double)b * (double)b;
            }
        }
        col_add(pbb, sh, a.bb, col, kv);
    UNIT_END
    if (!grid_sync(a.bar)) return;
    float* z = nullptr;
    if (!e0_vcycle(a.mg, a.bar, z)) return;
    UNIT_LOOP
        double prz = 0.0;
        if (kv) {
            NODE_LOOP
                const T zv = static_cast<T>(ldg2(z + em));
                a.P[e] = zv;
                prz += (double)ldg2(a.R + e) * (double)zv;
            }
        }
        col_add(prz, sh, slot(a, 2, 1), col, kv);
    UNIT_END
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        slot(a, 2, 2)[c] = ldg2(a.bb + c);
    if (!grid_sync(a.bar)) return;

    int it = 0;
    for (; it < a.maxit; ++it) {
        const int cur = it % 3, prev = (it + 2) % 3, next = (it + 1) % 3;
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < 3 * nc; c += blockDim.x)
                a.acc[(size_t)next * 3 * nc + c] = 0.0;
        // ---------------------------------- phase 1: AP = E_0 P, p.Ap
        UNIT_LOOP
            const bool act = kv && ldg2(slot(a, prev, 2) + col) > a.tol2 * ldg2(a.bb + col);
            double ppap = 0.0;
            if (act) {
                const T* Pr = a.P + (size_t)r * a.nRp * a.nSp;
                NODE_LOOP
                    T y = 0;
                    for (int p = a.st_ptr[i]; p < a.st_ptr[i + 1]; ++p)
                        y += __ldg(a.coef + (size_t)p * a.nSp + k) *
                             ldg2(Pr + (size_t)a.st_col[p] * a.nSp + k);
                    a.AP[e] = y;
                    ppap += (double)y * (double)ldg2(a.P + e);
                }
            }
            col_add(ppap, sh, slot(a, cur, 0), col, act);
        UNIT_END
        if (!grid_sync(a.bar)) return;
        // --------------------- phase 2: x, r update, rr, V-cycle input
        UNIT_LOOP
            const bool act = kv && ldg2(slot(a, prev, 2) + col) > a.tol2 * ldg2(a.bb + col);
            double prr = 0.0;
            if (kv) {
                const double pap = ldg2(slot(a, cur, 0) + col);
                const double alpha = (act && pap != 0.0) ? ldg2(slot(a, prev, 1) + col) / pap : 0.0;
                NODE_LOOP
                    if (act) {
                        a.X[e] += alpha * (double)ldg2(a.P + e);
                        const T rv = ldg2(a.R + e) - static_cast<T>(alpha) * ldg2(a.AP + e);
                        a.R[e] = rv;
                        prr += (double)rv * (double)rv;
                        B0[em] = static_cast<float>(rv);
                    } else {
                        B0[em] = 0.f;
                    }
                }
            }
            col_add(prr, sh, slot(a, cur, 2), col, act);
        UNIT_END
        if (!grid_sync(a.bar)) return;
        // ------------------------------------------ z = V-cycle(r)
        if (!e0_vcycle(a.mg, a.bar, z)) return;
        // ------------------------------------------------- r.z
        UNIT_LOOP
            const bool act = kv && ldg2(slot(a, prev, 2) + col) > a.tol2 * ldg2(a.bb + col);
            double prz = 0.0;
            if (act) {
                NODE_LOOP
                    prz += (double)ldg2(a.R + e) * (double)ldg2(z + em);
                }
            }
            col_add(prz, sh, slot(a, cur, 1), col, act);
        UNIT_END
        if (!grid_sync(a.bar)) return;
        // ---------------------------------------- p = z + beta p
        UNIT_LOOP
            if (!kv) continue;
            const bool was = ldg2(slot(a, prev, 2) + col) > a.tol2 * ldg2(a.bb + col);
            if (!was) {
                if (chunk == 0 && ny == 0) {
                    slot(a, cur, 2)[col] = ldg2(slot(a, prev, 2) + col);
                    slot(a, cur, 1)[col] = ldg2(slot(a, prev, 1) + col);
                }
                continue;
            }
            if (!(ldg2(slot(a, cur, 2) + col) > a.tol2 * ldg2(a.bb + col))) continue;
            const double rzo = ldg2(slot(a, prev, 1) + col);
            const double beta = rzo != 0.0 ? ldg2(slot(a, cur, 1) + col) / rzo : 0.0;
            NODE_LOOP
                a.P[e] = static_cast<T>(ldg2(z + em)) + static_cast<T>(beta) * ldg2(a.P + e);
            }
        UNIT_END
        if (!grid_sync(a.bar)) return;
        if (threadIdx.x == 0) s_stop = 1;
        __syncthreads();
        for (int c = threadIdx.x; c < nc; c += blockDim.x)
            if (ldg2(slot(a, cur, 2) + c) > a.tol2 * ldg2(a.bb + c)) s_stop = 0;
        __syncthreads();
        if (s_stop) {
            ++it;
            break;
        }
    }
#undef UNIT_LOOP
#undef UNIT_END
#undef NODE_LOOP
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status->iterations = it;
        a.status->converged = s_stop;
    }
}

// ============================================================ E_c V-cycle
struct EcLevel {
    int n;
    const int *ptr, *col;
    const float* val;      // [nnz][d][d]
    const float* dinv;     // [n][d][d]
    const int *rptr, *ridx, *p0, *p1;
    const float *rw, *w0, *w1;
    float *X, *Xt, *B;     // [nrhs][n][d]
};

struct EcMG {
    int L, nrhs, d, nu;
    bool dense;
    const float* cinv;     // [(n_c d)][(n_c d)]
    EcLevel lev[kMaxMGLevels];
};

// warp-level loop over (rhs, node) pairs of a level; lane = mode
#define WARP_LOOP(nn)                                                              \
    for (size_t wi = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;         \
         wi < (size_t)mg.nrhs * (nn); wi += ((size_t)gridDim.x * blockDim.x) >> 5) { \
        const int r = (int)(wi / (nn)), i = (int)(wi % (nn));                      \
        const size_t base = ((size_t)r * (nn) + i) * d;

__device__ __forceinline__ float ec_apply(const EcLevel& L, const float* x, int r, int i, int d,
                                          int lane) {
    float y = 0.f;
    if (lane < d)
        for (int p = L.ptr[i]; p < L.ptr[i + 1]; ++p) {
            const float* blk = L.val + ((size_t)p * d + lane) * d;
            const float* xv = x + ((size_t)r * L.n + L.col[p]) * d;
            for (int b = 0; b < d; ++b) y += __ldg(blk + b) * ldg2(xv + b);
        }
    return y;
}

__device__ __forceinline__ float ec_dmul(const float* D, int d, float v, int lane) {
    float y = 0.f;
    for (int b = 0; b < d; ++b) {
        const float vb = __shfl_sync(0xffffffffu, v, b);
        if (lane < d) y += __ldg(D + lane * d + b) * vb;
    }
    return y;
}

__device__ bool ec_vcycle(const EcMG& mg, GridBar* bar, float*& z) {
    const int d = mg.d;
    const int lane = threadIdx.x & 31;
    int cur[kMaxMGLevels];
    for (int l = 0; l < mg.L; ++l) cur[l] = 0;
    auto buf = [&](int l, int which) { return which ? mg.lev[l].Xt : mg.lev[l].X; };
    auto jacobi = [&](int l) -> bool {
        const EcLevel& Lv = mg.lev[l];
        const float* x = buf(l, cur[l]);
        float* xt = buf(l, cur[l] ^ 1);
        WARP_LOOP(Lv.n)
            const float y = ec_apply(Lv, x, r, i, d, lane);
            const float res = lane < d ? ldg2(Lv.B + base + lane) - y : 0.f;
            const float dx = ec_dmul(Lv.dinv + (size_t)i * d * d, d, res, lane);
            if (lane < d) xt[base + lane] = ldg2(x + base + lane) + kOmega * dx;
        }
        cur[l] ^= 1;
        return grid_sync(bar);
    };
    auto first = [&](int l) -> bool {
        const EcLevel& Lv = mg.lev[l];
        float* x = buf(l, 0);
        WARP_LOOP(Lv.n)
            const float bv = lane < d ? ldg2(Lv.B + base + lane) : 0.f;
            const float dx = ec_dmul(Lv.dinv + (size_t)i * d * d, d, bv, lane);
            if (lane < d) x[base + lane] = kOmega * dx;
        }
        cur[l] = 0;
        return grid_sync(bar);
    };
    for (int l = 0; l + 1 < mg.L; ++l) {
        const EcLevel& Lv = mg.lev[l];
        if (!first(l)) return false;
        for (int k = 1; k < mg.nu; ++k)
            if (!jacobi(l)) return false;
        const float* x = buf(l, cur[l]);
        float* t = buf(l, cur[l] ^ 1);
        WARP_LOOP(Lv.n)
            const float y = ec_apply(Lv, x, r, i, d, lane);
            if (lane < d) t[base + lane] = ldg2(Lv.B + base + lane) - y;
        }
        if (!grid_sync(bar)) return false;
        const EcLevel& Cv = mg.lev[l + 1];
        WARP_LOOP(Cv.n)
            if (lane < d) {
                float acc = 0.f;
                for (int q = Lv.rptr[i]; q < Lv.rptr[i + 1]; ++q)
                    acc += Lv.rw[q] * ldg2(t + ((size_t)r * Lv.n + Lv.ridx[q]) * d + lane);
                Cv.B[base + lane] = acc;
            }
        }
        if (!grid_sync(bar)) return false;
    }
    {
        const int l = mg.L - 1;
        const EcLevel& Lv = mg.lev[l];
        if (mg.dense) {
            float* x = buf(l, 0);
            const int N = Lv.n * d;
            WARP_LOOP(Lv.n)
                if (lane < d) {
                    const float* row = mg.cinv + (size_t)(i * d + lane) * N;
                    const float* b = Lv.B + (size_t)r * N;
                    float acc = 0.f;
                    for (int j = 0; j < N; ++j) acc += __ldg(row + j) * ldg2(b + j);
                    x[base + lane] = acc;
                }
            }
            cur[l] = 0;
            if (!grid_sync(bar)) return false;
        } else {
            if (!first(l)) return false;
            for (int k = 1; k < kCoarseSweeps; ++k)
                if (!jacobi(l)) return false;
        }
    }
    for (int l = mg.L - 2; l >= 0; --l) {
        const EcLevel& Lv = mg.lev[l];
        float* x = buf(l, cur[l]);
        const float* xc = buf(l + 1, cur[l + 1]);
        const int ncn = mg.lev[l + 1].n;
        WARP_LOOP(Lv.n)
            if (lane < d) {
                float v = Lv.w0[i] * ldg2(xc + ((size_t)r * ncn + Lv.p0[i]) * d + lane);
                if (Lv.p1[i] >= 0) v += Lv.w1[i] * ldg2(xc + ((size_t)r * ncn + Lv.p1[i]) * d + lane);
                x[base + lane] = ldg2(x + base + lane) + v;
            }
        }
        if (!grid_sync(bar)) return false;
        for (int k = 0; k < mg.nu; ++k)
            if (!jacobi(l)) return false;
    }
    z = buf(0, cur[0]);
    return true;
}

// ============================================================== E_c PCG
struct EcArgs {
    int nRp, d, nrhs, maxit;
    double tol2;
    const int* st_ptr;
    const int* st_col;
    const double* ec;   // FP64 blocks of E_c
    const double* B;
    double* X;
    double* R;
    double* P;
    double* AP;
    double* acc;        // [3][3][nrhs]
    double* bb;
    GridBar* bar;
    SolveStatus* status;
    EcMG mg;
};

__device__ void rhs_add(double v, double* sh, double* dst, int r) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(dst + r, v);
}

__global__ void __launch_bounds__(256) k_ec_pcg(EcArgs a) {
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = 0;
    const int d = a.d;
    const int lane = threadIdx.x & 31;
    const EcMG& mg = a.mg;
    float* B0 = mg.lev[0].B;
    auto sl = [&](int s, int q) { return a.acc + ((size_t)s * 3 + q) * a.nrhs; };
    WARP_LOOP(a.nRp)
        double pbb = 0.0;
        if (lane < d) {
            const double b = a.B[base + lane];
            a.X[base + lane] = 0.0;
            a.R[base + lane] = b;
            B0[base + lane] = (float)b;
            pbb = b * b;
        }
        rhs_add(pbb, nullptr, a.bb, r);
    }
    if (!grid_sync(a.bar)) return;
    float* z = nullptr;
    if (!ec_vcycle(mg, a.bar, z)) return;
    WARP_LOOP(a.nRp)
        double prz = 0.0;
        if (lane < d) {
            const double zv = ldg2(z + base + lane);
            a.P[base + lane] = zv;
            prz = ldg2(a.R + base + lane) * zv;
        }
        rhs_add(prz, nullptr, sl(2, 1), r);
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nrhs; c += gridDim.x * blockDim.x)
        sl(2, 2)[c] = ldg2(a.bb + c);
    if (!grid_sync(a.bar)) return;
    int it = 0;
    for (; it < a.maxit; ++it) {
        const int cur = it % 3, prev = (it + 2) % 3, next = (it + 1) % 3;
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < 3 * a.nrhs; c += blockDim.x)
                a.acc[(size_t)next * 3 * a.nrhs + c] = 0.0;
        WARP_LOOP(a.nRp)
            const bool act = ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
            if (!act) continue;
            double y = 0.0;
            if (lane < d)
                for (int p = a.st_ptr[i]; p < a.st_ptr[i + 1]; ++p) {
                    const double* blk = a.ec + ((size_t)p * d + lane) * d;
                    const double* xv = a.P + ((size_t)r * a.nRp + a.st_col[p]) * d;
                    for (int b = 0; b < d; ++b) y = fma(__ldg(blk + b), ldg2(xv + b), y);
                }
            double ppap = 0.0;
            if (lane < d) {
                a.AP[base + lane] = y;
                ppap = y * ldg2(a.P + base + lane);
            }
            rhs_add(ppap, nullptr, sl(cur, 0), r);
        }
        if (!grid_sync(a.bar)) return;
        WARP_LOOP(a.nRp)
            const bool act = ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
            double prr = 0.0;
            if (act && lane < d) {
                const double pap = ldg2(sl(cur, 0) + r);
                const double alpha = pap != 0.0 ? ldg2(sl(prev, 1) + r) / pap : 0.0;
                a.X[base + lane] += alpha * ldg2(a.P + base + lane);
                const double rv = ldg2(a.R + base + lane) - alpha * ldg2(a.AP + base + lane);
                a.R[base + lane] = rv;
                prr = rv * rv;
                B0[base + lane] = (float)rv;
            } else if (lane < d) {
                B0[base + lane] = 0.f;
            }
            if (act) rhs_add(prr, nullptr, sl(cur, 2), r);
        }
        if (!grid_sync(a.bar)) return;
        if (!ec_vcycle(mg, a.bar, z)) return;
        WARP_LOOP(a.nRp)
            const bool act = ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
            if (!act) continue;
            double prz = 0.0;
            if (lane < d) prz = ldg2(a.R + base + lane) * (double)ldg2(z + base + lane);
            rhs_add(prz, nullptr, sl(cur, 1), r);
        }
        if (!grid_sync(a.bar)) return;
        WARP_LOOP(a.nRp)
            const bool was = ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
            if (!was) {
                if (i == 0 && lane == 0) {
                    sl(cur, 2)[r] = ldg2(sl(prev, 2) + r);
                    sl(cur, 1)[r] = ldg2(sl(prev, 1) + r);
                }
                continue;
            }
            if (!(ldg2(sl(cur, 2) + r) > a.tol2 * ldg2(a.bb + r)) || lane >= d) continue;
            const double rzo = ldg2(sl(prev, 1) + r);
            const double beta = rzo != 0.0 ? ldg2(sl(cur, 1) + r) / rzo : 0.0;
            a.P[base + lane] = (double)ldg2(z + base + lane) + beta * ldg2(a.P + base + lane);
        }
        if (!grid_sync(a.bar)) return;
        if (threadIdx.x == 0) s_stop = 1;
        __syncthreads();
        for (int c = threadIdx.x; c < a.nrhs; c += blockDim.x)
            if (ldg2(sl(cur, 2) + c) > a.tol2 * ldg2(a.bb + c)) s_stop = 0;
        __syncthreads();
        if (s_stop) {
            ++it;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status->iterations = it;
        a.status->converged = s_stop;
    }
}
#undef WARP_LOOP

__global__ void k_copy_err(const GridBar* bar, SolveStatus* st) { st->timed_out = bar->err; }

int coop_grid(const void* fn, int threads, int cap_blocks) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    per_sm = std::max(1, std::min(per_sm, 2));
    return std::max(1, std::min(per_sm * device_sm_count(), cap_blocks));
}

E0MG e0_mg_view(const MGDevice& m, int ncols, int nSp) {
    E0MG g{};
    g.L = m.L;
    g.ncols = ncols;
    g.nSp = nSp;
    g.nu = m.nu;
    g.dense = m.dense;
    g.cinv = m.cinv;
    g.e0s = m.e0s;
    for (int l = 0; l < m.L; ++l) {
        const MGDeviceLevel& s = m.lev[l];
        E0Level& t = g.lev[l];
        t.n = s.n; t.ptr = s.ptr; t.col = s.col; t.diag = s.diag; t.val = s.val; t.nnz = s.nnz;
        t.rptr = s.rptr; t.ridx = s.ridx; t.p0 = s.p0; t.p1 = s.p1;
        t.rw = s.rw; t.w0 = s.w0; t.w1 = s.w1;
        t.X = s.X; t.Xt = s.Xt; t.B = s.B;
    }
    return g;
}

EcMG ec_mg_view(const MGDevice& m, int nrhs, int d) {
    EcMG g{};
    g.L = m.L;
    g.nrhs = nrhs;
    g.d = d;
    g.nu = m.nu;
    g.dense = m.dense;
    g.cinv = m.cinv;
    for (int l = 0; l < m.L; ++l) {
        const MGDeviceLevel& s = m.lev[l];
        EcLevel& t = g.lev[l];
        t.n = s.n; t.ptr = s.ptr; t.col = s.col; t.val = s.val; t.dinv = s.dinv;
        t.rptr = s.rptr; t.ridx = s.ridx; t.p0 = s.p0; t.p1 = s.p1;
        t.rw = s.rw; t.w0 = s.w0; t.w1 = s.w1;
        t.X = s.X; t.Xt = s.Xt; t.B = s.B;
    }
    return g;
}

template <typename T>
int e0_pcg_impl(cudaStream_t s, const DevSystem& d, const T* coef, const double* B, double* X,
                int nrhs, double tol, int maxit, void* work, size_t work_bytes,
                SolveStatus* status_dev) {
    if (work_bytes < e0_cg_work_bytes(d, nrhs))
        return fail(RTE_ERR_ARG, "E_0 CG workspace too small");
    if (nrhs > d.e0mg.cap_cols / d.nSp) return fail(RTE_ERR_ARG, "E_0 multigrid sized for fewer RHS");
    const size_t n = (size_t)nrhs * d.nRp * d.nSp;
    const int ncols = nrhs * d.nSp;
    char* p = static_cast<char*>(work);
    E0Args<T> a;
    a.R = reinterpret_cast<T*>(carve<double>(p, n));
    a.P = reinterpret_cast<T*>(carve<double>(p, n));
    a.AP = reinterpret_cast<T*>(carve<double>(p, n));
    a.acc = carve<double>(p, 9 * (size_t)ncols);
    a.bb = carve<double>(p, ncols);
    a.bar = carve<GridBar>(p, 1);
    RTE_CUDA_TRY(cudaMemsetAsync(a.acc, 0, 9 * (size_t)ncols * 8, s));
    RTE_CUDA_TRY(cudaMemsetAsync(a.bb, 0, (size_t)ncols * 8, s));
    RTE_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(GridBar), s));
    RTE_CUDA_TRY(cudaMemsetAsync(status_dev, 0, sizeof(SolveStatus), s));
    a.nRp = d.nRp;
    a.nSp = d.nSp;
    a.nrhs = nrhs;
    a.ncols = ncols;
    a.kTiles = (d.nSp + 31) / 32;
    a.chunks = (d.nRp + kChunk - 1) / kChunk;
    a.units = nrhs * a.kTiles * a.chunks;
    a.maxit = maxit;
    a.tol2 = tol * tol;
    a.st_ptr = d.st_ptr;
    a.st_col = d.st_col;
    a.coef = coef;
    a.B = B;
    a.X = X;
    a.status = status_dev;
    a.mg = e0_mg_view(d.e0mg, ncols, d.nSp);
    const void* fn = (const void*)k_e0_pcg<T>;
    const int grid = coop_grid(fn, 256, 1 << 20);
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel(fn, grid, 256, args, 0, s));
    k_copy_err<<<1, 1, 0, s>>>(a.bar, status_dev);
    count_launches(2);
    return RTE_OK;
}

}  // namespace

size_t e0_cg_work_bytes(const DevSystem& d, int nrhs) {
    const size_t n = (size_t)nrhs * d.nRp * d.nSp;
    const size_t ncols = (size_t)nrhs * d.nSp;
    return 3 * (((n * 8) + 255) / 256 * 256) + ((9 * ncols * 8 + 255) / 256 * 256) +
           ((ncols * 8 + 255) / 256 * 256) + 256;
}

int e0_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs, double tol,
          int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    return e0_pcg_impl<double>(s, d, d.e0coef, B, X, nrhs, tol, maxit, work, work_bytes,
                               status_dev);
}

int e0_cg_lo(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
             double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    return e0_pcg_impl<float>(s, d, d.e0coef_f, B, X, nrhs, tol, maxit, work, work_bytes,
                              status_dev);
}

size_t coarse_cg_work_bytes(const DevSystem& d, int nrhs) {
    const size_t n = (size_t)nrhs * d.nRp * d.dP;
    return 3 * (((n * 8) + 255) / 256 * 256) + ((9 * (size_t)nrhs * 8 + 255) / 256 * 256) +
           (((size_t)nrhs * 8 + 255) / 256 * 256) + 256;
}

int coarse_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
              double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    if (d.dP < 1 || d.dP > 32) return fail(RTE_ERR_ARG, "coarse CG supports 1 <= d^+ <= 32");
    if (work_bytes < coarse_cg_work_bytes(d, nrhs))
        return fail(RTE_ERR_ARG, "coarse CG workspace too small");
    if (nrhs > d.ecmg.cap_cols) return fail(RTE_ERR_ARG, "coarse multigrid sized for fewer RHS");
    const size_t n = (size_t)nrhs * d.nRp * d.dP;
    char* p = static_cast<char*>(work);
    EcArgs a;
    a.R = carve<double>(p, n);
    a.P = carve<double>(p, n);
    a.AP = carve<double>(p, n);
    a.acc = carve<double>(p, 9 * (size_t)nrhs);
    a.bb = carve<double>(p, nrhs);
    a.bar = carve<GridBar>(p, 1);
    RTE_CUDA_TRY(cudaMemsetAsync(a.acc, 0, 9 * (size_t)nrhs * 8, s));
    RTE_CUDA_TRY(cudaMemsetAsync(a.bb, 0, (size_t)nrhs * 8, s));
    RTE_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(GridBar), s));
    RTE_CUDA_TRY(cudaMemsetAsync(status_dev, 0, sizeof(SolveStatus), s));
    a.nRp = d.nRp;
    a.d = d.dP;
    a.nrhs = nrhs;
    a.maxit = maxit;
    a.tol2 = tol * tol;
    a.st_ptr = d.st_ptr;
    a.st_col = d.st_col;
    a.ec = d.ec_val;
    a.B = B;
    a.X = X;
    a.status = status_dev;
    a.mg = ec_mg_view(d.ecmg, nrhs, d.dP);
    const void* fn = (const void*)k_ec_pcg;
    const int grid = coop_grid(fn, 256, 1 << 20);
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel(fn, grid, 256, args, 0, s));
    k_copy_err<<<1, 1, 0, s>>>(a.bar, status_dev);
    count_launches(2);
    return RTE_OK;
}

}  // namespace rte
