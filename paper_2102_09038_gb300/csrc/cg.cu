// Persistent conjugate-gradient kernels:
//  * E_0^{-1}: the n_S^+ decoupled direction blocks of
//    E_0 = (1-cg)^{-1} A^T (M^-)^{-1} A + R + M^+ (eq. equivalence_bE_bE0),
//    all (rhs, direction) columns in one launch, Jacobi preconditioned, each
//    column stopping on its own relative residual (Section 5.5 "E_0 is block
//    diagonal with n_S^+ sparse blocks").
//  * E_c^{-1}: the coarse Galerkin system of Section 5.4 with block-Jacobi
//    (d x d node blocks) preconditioning, one CG per right-hand side.
//
// Both run as one cooperative launch whose blocks meet at a grid barrier with
// a bounded wait: a barrier that does not complete within ~2 s sets an error
// flag and every block returns, so a fault shows up as RTE_ERR_TIMEOUT on the
// host instead of a hung GPU.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.h"
#include "rte_internal.h"

namespace rte {

namespace {

struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

constexpr unsigned long long kSpinLimit = 1ull << 24;

__device__ bool grid_sync(GridBar* gb) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &gb->gen;
        volatile int* verr = &gb->err;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gb->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == g) {
                __nanosleep(128);
                if (*verr) break;
                if (++spins > kSpinLimit) {
                    atomicExch(&gb->err, 1);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int*)&gb->err) == 0;
}

__device__ __forceinline__ double ld(const double* p) { return __ldcg(p); }

// ------------------------------------------------------------ E_0 CG
struct E0Args {
    int nRp, nSp, nrhs, nnz, ncols, kTiles, chunks, units, maxit;
    double tol2;
    const int* st_ptr;
    const int* st_col;
    const int* st_diag;
    const double* sval;
    const double* e0s;
    const double* B;
    double* X;
    double* R;
    double* P;
    double* AP;
    double* acc;   // [3 slots][3 quantities][ncols]: pAp, rz, rr
    double* bb;    // [ncols]
    GridBar* bar;
    SolveStatus* status;
};

constexpr int kE0Chunk = 64;   // nodes per work unit
constexpr int kE0Rows = 8;     // node rows per pass (blockDim.y)

__device__ __forceinline__ double e0_coef(const double* s, const double* sv, int nnz,
                                          int p) {
    return s[0] * sv[(size_t)kK11 * nnz + p] + s[1] * sv[(size_t)kK12 * nnz + p] +
           s[2] * sv[(size_t)kK22 * nnz + p] + s[3] * sv[(size_t)kBx * nnz + p] +
           s[4] * sv[(size_t)kBy * nnz + p] + s[5] * sv[(size_t)kMt * nnz + p];
}

__device__ __forceinline__ double* accp(const E0Args& a, int slot, int q) {
    return a.acc + ((size_t)slot * 3 + q) * a.ncols;
}

// Reduce a per-thread partial over the node rows of the block and add it
// to dst[col] (one atomic per column per unit).
__device__ void col_reduce_add(double v, double* sh, double* dst, int col, bool valid) {
    const int kx = threadIdx.x & 31, ny = threadIdx.x >> 5;
    sh[ny * 32 + kx] = v;
    __syncthreads();
    if (ny == 0) {
        double s = 0.0;
        for (int y = 0; y < kE0Rows; ++y) s += sh[y * 32 + kx];
        if (valid) atomicAdd(dst + col, s);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_e0_cg(E0Args a) {
    __shared__ double sh[kE0Rows * 32];
    __shared__ int s_stop;
    const int kx = threadIdx.x & 31, ny = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_stop = 0;
    // ---------------------------------------------------------------- init
    for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
        const int chunk = u % a.chunks;
        const int kt = (u / a.chunks) % a.kTiles;
        const int r = u / (a.chunks * a.kTiles);
        const int k = kt * 32 + kx;
        const bool kv = k < a.nSp;
        const int col = r * a.nSp + k;
        double s[6];
        for (int q = 0; q < 6; ++q) s[q] = kv ? a.e0s[6 * k + q] : 0.0;
        double prz = 0.0, pbb = 0.0;
        for (int t = 0; t < kE0Chunk / kE0Rows; ++t) {
            const int i = chunk * kE0Chunk + ny + kE0Rows * t;
            if (!kv || i >= a.nRp) continue;
            const size_t e = ((size_t)r * a.nRp + i) * a.nSp + k;
            const double b = a.B[e];
            const double dinv = 1.0 / e0_coef(s, a.sval, a.nnz, a.st_diag[i]);
            a.X[e] = 0.0;
            a.R[e] = b;
            a.P[e] = dinv * b;
            prz += b * dinv * b;
            pbb += b * b;
        }
        col_reduce_add(prz, sh, accp(a, 2, 1), col, kv);
        col_reduce_add(pbb, sh, a.bb, col, kv);
    }
    if (!grid_sync(a.bar)) return;
    // rr of the initial residual equals bb
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ncols;
         c += gridDim.x * blockDim.x)
        accp(a, 2, 2)[c] = ld(a.bb + c);
    if (!grid_sync(a.bar)) return;

    int it = 0;
    for (; it < a.maxit; ++it) {
        const int cur = it % 3, prev = (it + 2) % 3, next = (it + 1) % 3;
        // ------------------------------------------- phase 1: AP = E_0 P
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < 3 * a.ncols; c += blockDim.x)
                a.acc[(size_t)next * 3 * a.ncols + c] = 0.0;
        for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int chunk = u % a.chunks;
            const int kt = (u / a.chunks) % a.kTiles;
            const int r = u / (a.chunks * a.kTiles);
            const int k = kt * 32 + kx;
            const bool kv = k < a.nSp;
            const int col = r * a.nSp + k;
            const bool act = kv && ld(accp(a, prev, 2) + col) > a.tol2 * ld(a.bb + col);
            double s[6];
            for (int q = 0; q < 6; ++q) s[q] = kv ? a.e0s[6 * k + q] : 0.0;
            double ppap = 0.0;
            if (act) {
                const double* Pr = a.P + (size_t)r * a.nRp * a.nSp;
                for (int t = 0; t < kE0Chunk / kE0Rows; ++t) {
                    const int i = chunk * kE0Chunk + ny + kE0Rows * t;
                    if (i >= a.nRp) continue;
                    double y = 0.0;
                    for (int p = a.st_ptr[i]; p < a.st_ptr[i + 1]; ++p)
                        y += e0_coef(s, a.sval, a.nnz, p) *
                             ld(Pr + (size_t)a.st_col[p] * a.nSp + k);
                    const size_t e = ((size_t)r * a.nRp + i) * a.nSp + k;
                    a.AP[e] = y;
                    ppap += y * ld(Pr + (size_t)i * a.nSp + k);
                }
            }
            col_reduce_add(ppap, sh, accp(a, cur, 0), col, act);
        }
        if (!grid_sync(a.bar)) return;
        // ------------------------------- phase 2: x, r update; rz, rr
        for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int chunk = u % a.chunks;
            const int kt = (u / a.chunks) % a.kTiles;
            const int r = u / (a.chunks * a.kTiles);
            const int k = kt * 32 + kx;
            const bool kv = k < a.nSp;
            const int col = r * a.nSp + k;
            const bool act = kv && ld(accp(a, prev, 2) + col) > a.tol2 * ld(a.bb + col);
            double s[6];
            for (int q = 0; q < 6; ++q) s[q] = kv ? a.e0s[6 * k + q] : 0.0;
            double prz = 0.0, prr = 0.0;
            if (act) {
                const double pap = ld(accp(a, cur, 0) + col);
                const double alpha = pap != 0.0 ? ld(accp(a, prev, 1) + col) / pap : 0.0;
                for (int t = 0; t < kE0Chunk / kE0Rows; ++t) {
                    const int i = chunk * kE0Chunk + ny + kE0Rows * t;
                    if (i >= a.nRp) continue;
                    const size_t e = ((size_t)r * a.nRp + i) * a.nSp + k;
                    a.X[e] += alpha * ld(a.P + e);
                    const double rv = ld(a.R + e) - alpha * ld(a.AP + e);
                    a.R[e] = rv;
                    const double dinv = 1.0 / e0_coef(s, a.sval, a.nnz, a.st_diag[i]);
                    prz += rv * dinv * rv;
                    prr += rv * rv;
                }
            }
            col_reduce_add(prz, sh, accp(a, cur, 1), col, act);
            col_reduce_add(prr, sh, accp(a, cur, 2), col, act);
        }
        if (!grid_sync(a.bar)) return;
        // -------------------------------------- phase 3: p = z + beta p
        for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int chunk = u % a.chunks;
            const int kt = (u / a.chunks) % a.kTiles;
            const int r = u / (a.chunks * a.kTiles);
            const int k = kt * 32 + kx;
            const bool kv = k < a.nSp;
            const int col = r * a.nSp + k;
            const bool was = kv && ld(accp(a, prev, 2) + col) > a.tol2 * ld(a.bb + col);
            if (!was) {
                // keep the stopping state: carry rr and rz forward
                if (kv && chunk == 0 && ny == 0) {
                    accp(a, cur, 2)[col] = ld(accp(a, prev, 2) + col);
                    accp(a, cur, 1)[col] = ld(accp(a, prev, 1) + col);
                }
                continue;
            }
            const bool act = ld(accp(a, cur, 2) + col) > a.tol2 * ld(a.bb + col);
            if (!act) continue;
            double s[6];
            for (int q = 0; q < 6; ++q) s[q] = a.e0s[6 * k + q];
            const double rzo = ld(accp(a, prev, 1) + col);
            const double beta = rzo != 0.0 ? ld(accp(a, cur, 1) + col) / rzo : 0.0;
            for (int t = 0; t < kE0Chunk / kE0Rows; ++t) {
                const int i = chunk * kE0Chunk + ny + kE0Rows * t;
                if (i >= a.nRp) continue;
                const size_t e = ((size_t)r * a.nRp + i) * a.nSp + k;
                const double dinv = 1.0 / e0_coef(s, a.sval, a.nnz, a.st_diag[i]);
                a.P[e] = dinv * ld(a.R + e) + beta * ld(a.P + e);
            }
        }
        if (!grid_sync(a.bar)) return;
        // ----------------------------------------- all columns converged?
        if (threadIdx.x == 0) s_stop = 1;
        __syncthreads();
        for (int c = threadIdx.x; c < a.ncols; c += blockDim.x)
            if (ld(accp(a, cur, 2) + c) > a.tol2 * ld(a.bb + c)) s_stop = 0;
        __syncthreads();
        if (s_stop) {
            ++it;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status->iterations = it;
        a.status->converged = it < a.maxit || s_stop;
    }
}

// ---------------------------------------------------------- coarse CG
struct CoarseArgs {
    int nRp, d, nrhs, chunks, units, maxit;
    double tol2;
    const int* st_ptr;
    const int* st_col;
    const double* ec;
    const double* dinv;
    const double* B;
    double* X;
    double* R;
    double* P;
    double* AP;
    double* Z;
    double* acc;   // [3 slots][3][nrhs]
    double* bb;    // [nrhs]
    GridBar* bar;
    SolveStatus* status;
};

constexpr int kCoNodes = 8;   // nodes per unit (one warp per node)

// y[i][a] = sum_b D[a][b] x[b] across the lanes of one warp (lane = a)
__device__ __forceinline__ double warp_block_apply(const double* Dblk, int d, double xa,
                                                   int lane) {
    double y = 0.0;
    for (int b = 0; b < d; ++b) {
        const double xb = __shfl_sync(0xffffffffu, xa, b);
        if (lane < d) y = fma(Dblk[lane * d + b], xb, y);
    }
    return y;
}

__device__ void rhs_reduce_add(double v, double* sh, double* dst, int r) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int y = 0; y < kCoNodes; ++y) s += sh[y];
        atomicAdd(dst + r, s);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_coarse_cg(CoarseArgs a) {
    __shared__ double sh[kCoNodes];
    __shared__ int s_stop;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_stop = 0;
    auto accp = [&](int slot, int q) { return a.acc + ((size_t)slot * 3 + q) * a.nrhs; };
    for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
        const int chunk = u % a.chunks, r = u / a.chunks;
        const int i = chunk * kCoNodes + w;
        double prz = 0.0, pbb = 0.0;
        if (i < a.nRp) {
            const size_t e = ((size_t)r * a.nRp + i) * a.d + lane;
            const double b = lane < a.d ? a.B[e] : 0.0;
            const double z = warp_block_apply(a.dinv + (size_t)i * a.d * a.d, a.d, b, lane);
            if (lane < a.d) {
                a.X[e] = 0.0;
                a.R[e] = b;
                a.P[e] = z;
                prz = b * z;
                pbb = b * b;
            }
        }
        rhs_reduce_add(prz, sh, accp(2, 1), r);
        rhs_reduce_add(pbb, sh, a.bb, r);
    }
    if (!grid_sync(a.bar)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nrhs; c += gridDim.x * blockDim.x)
        accp(2, 2)[c] = ld(a.bb + c);
    if (!grid_sync(a.bar)) return;
    int it = 0;
    for (; it < a.maxit; ++it) {
        const int cur = it % 3, prev = (it + 2) % 3, next = (it + 1) % 3;
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < 3 * a.nrhs; c += blockDim.x)
                a.acc[(size_t)next * 3 * a.nrhs + c] = 0.0;
        for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int chunk = u % a.chunks, r = u / a.chunks;
            const bool act = ld(accp(prev, 2) + r) > a.tol2 * ld(a.bb + r);
            const int i = chunk * kCoNodes + w;
            double ppap = 0.0;
            if (act && i < a.nRp) {
                const double* Pr = a.P + (size_t)r * a.nRp * a.d;
                double y = 0.0;
                if (lane < a.d)
                    for (int p = a.st_ptr[i]; p < a.st_ptr[i + 1]; ++p) {
                        const double* blk = a.ec + ((size_t)p * a.d + lane) * a.d;
                        const double* xv = Pr + (size_t)a.st_col[p] * a.d;
                        for (int b = 0; b < a.d; ++b) y = fma(blk[b], ld(xv + b), y);
                    }
                if (lane < a.d) {
                    const size_t e = ((size_t)r * a.nRp + i) * a.d + lane;
                    a.AP[e] = y;
                    ppap = y * ld(a.P + e);
                }
            }
            if (act) rhs_reduce_add(ppap, sh, accp(cur, 0), r);
        }
        if (!grid_sync(a.bar)) return;
        for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int chunk = u % a.chunks, r = u / a.chunks;
            const bool act = ld(accp(prev, 2) + r) > a.tol2 * ld(a.bb + r);
            const int i = chunk * kCoNodes + w;
            double prz = 0.0, prr = 0.0;
            if (act && i < a.nRp) {
                const double pap = ld(accp(cur, 0) + r);
                const double alpha = pap != 0.0 ? ld(accp(prev, 1) + r) / pap : 0.0;
                const size_t e = ((size_t)r * a.nRp + i) * a.d + lane;
                double rv = 0.0;
                if (lane < a.d) {
                    a.X[e] += alpha * ld(a.P + e);
                    rv = ld(a.R + e) - alpha * ld(a.AP + e);
                    a.R[e] = rv;
                }
                const double z = warp_block_apply(a.dinv + (size_t)i * a.d * a.d, a.d, rv, lane);
                if (lane < a.d) {
                    a.Z[e] = z;
                    prz = rv * z;
                    prr = rv * rv;
                }
            }
            if (act) {
                rhs_reduce_add(prz, sh, accp(cur, 1), r);
                rhs_reduce_add(prr, sh, accp(cur, 2), r);
            }
        }
        if (!grid_sync(a.bar)) return;
        for (int u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int chunk = u % a.chunks, r = u / a.chunks;
            const bool was = ld(accp(prev, 2) + r) > a.tol2 * ld(a.bb + r);
            const int i = chunk * kCoNodes + w;
            if (!was) {
                if (chunk == 0 && threadIdx.x == 0) {
                    accp(cur, 2)[r] = ld(accp(prev, 2) + r);
                    accp(cur, 1)[r] = ld(accp(prev, 1) + r);
                }
                continue;
            }
            const bool act = ld(accp(cur, 2) + r) > a.tol2 * ld(a.bb + r);
            if (!act || i >= a.nRp || lane >= a.d) continue;
            const double rzo = ld(accp(prev, 1) + r);
            const double beta = rzo != 0.0 ? ld(accp(cur, 1) + r) / rzo : 0.0;
            const size_t e = ((size_t)r * a.nRp + i) * a.d + lane;
            a.P[e] = ld(a.Z + e) + beta * ld(a.P + e);
        }
        if (!grid_sync(a.bar)) return;
        if (threadIdx.x == 0) s_stop = 1;
        __syncthreads();
        for (int c = threadIdx.x; c < a.nrhs; c += blockDim.x)
            if (ld(accp(cur, 2) + c) > a.tol2 * ld(a.bb + c)) s_stop = 0;
        __syncthreads();
        if (s_stop) {
            ++it;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status->iterations = it;
        a.status->converged = it < a.maxit || s_stop;
    }
}

__global__ void k_copy_err(const GridBar* bar, SolveStatus* st) {
    st->timed_out = bar->err;
}

int cooperative_grid(const void* fn, int threads, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    per_sm = std::max(1, std::min(per_sm, 4));
    return per_sm * device_sm_count();
}

template <typename T>
T* carve(char*& p, size_t n) {
    T* out = reinterpret_cast<T*>(p);
    p += ((n * sizeof(T) + 255) / 256) * 256;
    return out;
}

}  // namespace

size_t e0_cg_work_bytes(const DevSystem& d, int nrhs) {
    const size_t n = (size_t)nrhs * d.nRp * d.nSp;
    const size_t ncols = (size_t)nrhs * d.nSp;
    return 3 * (((n * 8) + 255) / 256 * 256) + ((9 * ncols * 8 + 255) / 256 * 256) +
           ((ncols * 8 + 255) / 256 * 256) + 256;
}

int e0_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
          double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    if (work_bytes < e0_cg_work_bytes(d, nrhs))
        return fail(RTE_ERR_ARG, "E_0 CG workspace too small");
    const size_t n = (size_t)nrhs * d.nRp * d.nSp;
    const int ncols = nrhs * d.nSp;
    char* p = static_cast<char*>(work);
    E0Args a;
    a.R = carve<double>(p, n);
    a.P = carve<double>(p, n);
    a.AP = carve<double>(p, n);
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
    a.nnz = d.nnz;
    a.ncols = ncols;
    a.kTiles = (d.nSp + 31) / 32;
    a.chunks = (d.nRp + kE0Chunk - 1) / kE0Chunk;
    a.units = nrhs * a.kTiles * a.chunks;
    a.maxit = maxit;
    a.tol2 = tol * tol;
    a.st_ptr = d.st_ptr;
    a.st_col = d.st_col;
    a.st_diag = d.st_diag;
    a.sval = d.sval;
    a.e0s = d.e0s;
    a.B = B;
    a.X = X;
    a.status = status_dev;
    const int grid = std::min(cooperative_grid((const void*)k_e0_cg, 256, 0), a.units);
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_e0_cg, grid, 256, args, 0, s));
    k_copy_err<<<1, 1, 0, s>>>(a.bar, status_dev);
    count_launches(2);
    return RTE_OK;
}

size_t coarse_cg_work_bytes(const DevSystem& d, int nrhs) {
    const size_t n = (size_t)nrhs * d.nRp * d.dP;
    return 4 * (((n * 8) + 255) / 256 * 256) + ((9 * (size_t)nrhs * 8 + 255) / 256 * 256) +
           (((size_t)nrhs * 8 + 255) / 256 * 256) + 256;
}

int coarse_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
              double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    if (d.dP < 1 || d.dP > 32) return fail(RTE_ERR_ARG, "coarse CG supports 1 <= d^+ <= 32");
    if (work_bytes < coarse_cg_work_bytes(d, nrhs))
        return fail(RTE_ERR_ARG, "coarse CG workspace too small");
    const size_t n = (size_t)nrhs * d.nRp * d.dP;
    char* p = static_cast<char*>(work);
    CoarseArgs a;
    a.R = carve<double>(p, n);
    a.P = carve<double>(p, n);
    a.AP = carve<double>(p, n);
    a.Z = carve<double>(p, n);
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
    a.chunks = (d.nRp + kCoNodes - 1) / kCoNodes;
    a.units = nrhs * a.chunks;
    a.maxit = maxit;
    a.tol2 = tol * tol;
    a.st_ptr = d.st_ptr;
    a.st_col = d.st_col;
    a.ec = d.ec_val;
    a.dinv = d.ec_dinv;
    a.B = B;
    a.X = X;
    a.status = status_dev;
    const int grid = std::min(cooperative_grid((const void*)k_coarse_cg, 256, 0), a.units);
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_coarse_cg, grid, 256, args, 0, s));
    k_copy_err<<<1, 1, 0, s>>>(a.bar, status_dev);
    count_launches(2);
    return RTE_OK;
}

}  // namespace rte
