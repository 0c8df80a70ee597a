// Set-up of the direct route of the coarse solve E_c^{-1} (Section 5.4's
// coarse system, eq. corr_discrete): the inverses of the row Schur
// complements of E_c, which is block tridiagonal over the mesh rows y with
// row blocks of Bd = (m+1) d unknowns (node-major, component fastest):
//   S_0 = A_00,   S_y = A_yy - A_y,y-1 S_y-1^{-1} A_y-1,y,
// A_y,y-1 reaching the nodes (x, y-1) and (x-1, y-1) of the row below.
// Each S_y is formed in FP64 on the device from the stencil blocks and the
// previous row's inverse (two sparse-dense products), factorised and
// inverted by cuSOLVER (Cholesky, FP64), symmetrised and stored (FP32 for
// the mixed modes, FP64 for FP64 mode).  The sweeps that use it run inside
// the coarse CG kernel (mg.cu, ec_sweep).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <vector>

#include "device.h"
#include "rte_internal.h"

namespace rte {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(size_t n) {
    return (unsigned)std::min<size_t>((n + kThreads - 1) / kThreads, 65535u * 8u);
}

// entry (ra, cb) of the d x d stencil block of `node` in direction dir
// (blocks stored transposed: column cb, row ra)
__device__ __forceinline__ double blk(const double* ec, int n, int d, int dir, int node, int ra,
                                      int cb) {
    return ec[((size_t)dir * n + node) * d * d + (size_t)cb * d + ra];
}

// R = S_y-1^{-1} L^T with L = A_y,y-1: R[(u,c)][(x',a')] =
// sum_c' Sp[(u,c)][(x',c')] L4(x')[a'][c'] + Sp[(u,c)][(x'-1,c')] L6(x')[a'][c']
__global__ void k_ec_schur_r(int m, int d, int y, const double* __restrict__ ec,
                             const double* __restrict__ Sp, double* __restrict__ R) {
    const int b = m + 1, n = b * b, Bd = b * d;
    const size_t total = (size_t)Bd * Bd;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / Bd), col = (int)(e % Bd);
        const int xp = col / d, ap = col - xp * d, node = y * b + xp;
        const double* sr = Sp + (size_t)row * Bd;
        double s = 0.0;
        for (int c = 0; c < d; ++c) {
            s += sr[xp * d + c] * blk(ec, n, d, 4, node, ap, c);
            if (xp > 0) s += sr[(xp - 1) * d + c] * blk(ec, n, d, 6, node, ap, c);
        }
        R[e] = s;
    }
}

// S = A_yy - L R (y > 0), S = A_00 (y = 0); row-major Bd x Bd (symmetric, so
// also the column-major matrix cuSOLVER reads)
__global__ void k_ec_schur_s(int m, int d, int y, const double* __restrict__ ec,
                             const double* __restrict__ R, double* __restrict__ S) {
    const int b = m + 1, n = b * b, Bd = b * d;
    const size_t total = (size_t)Bd * Bd;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / Bd), col = (int)(e % Bd);
        const int x = row / d, a = row - x * d, xp = col / d, ap = col - xp * d;
        const int node = y * b + x;
        double v = 0.0;
        if (xp == x) v = blk(ec, n, d, 0, node, a, ap);
        else if (xp == x + 1) v = blk(ec, n, d, 1, node, a, ap);
        else if (xp == x - 1) v = blk(ec, n, d, 2, node, a, ap);
        if (y > 0) {
            for (int c = 0; c < d; ++c) {
                v -= blk(ec, n, d, 4, node, a, c) * R[(size_t)(x * d + c) * Bd + col];
                if (x > 0) v -= blk(ec, n, d, 6, node, a, c) * R[(size_t)((x - 1) * d + c) * Bd + col];
            }
        }
        S[e] = v;
    }
}

// The inverse cuSOLVER left in the lower triangle (column-major) of Si:
// symmetrised into the FP64 scratch Sp (the next row's input) and the factor
// row y ([Bd][ldf], FP32 or FP64).
__global__ void k_ec_store(int Bd, int ldf, const double* __restrict__ Si, double* __restrict__ Sp,
                           float* __restrict__ f32, double* __restrict__ f64) {
    const size_t total = (size_t)Bd * ldf;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldf), j = (int)(e % ldf);
        double v = 0.0;
        if (j < Bd) {
            // column-major lower triangle: (i, j) with i >= j at i + j Bd
            v = i >= j ? Si[(size_t)i + (size_t)j * Bd] : Si[(size_t)j + (size_t)i * Bd];
            Sp[(size_t)i * Bd + j] = v;
        }
        if (f32) f32[e] = (float)v;
        if (f64) f64[e] = v;
    }
}

}  // namespace

int ec_direct_ld(int m, int d) { return ((m + 1) * d + 3) & ~3; }

size_t ec_direct_bytes(int m, int d, bool fp64) {
    const size_t Bd = (size_t)(m + 1) * d;
    return (size_t)(m + 1) * Bd * ec_direct_ld(m, d) * (fp64 ? 8 : 4);
}

bool ec_direct_fits(int m, int d) { return m >= 1 && (m + 1) * d <= 2400; }

int ec_direct_factor(cudaStream_t s, void* solver, const DevSystem& d, float* out32,
                     double* out64) {
    const int m = d.m, dP = d.dP, Bd = (m + 1) * dP, ldf = ec_direct_ld(m, dP);
    if (!ec_direct_fits(m, dP)) return fail(RTE_ERR_ARG, "coarse system too large for the direct route");
    cusolverDnHandle_t cs = static_cast<cusolverDnHandle_t>(solver);
    const size_t bb = (size_t)Bd * Bd;
    double *Sp = nullptr, *R = nullptr, *S = nullptr, *work = nullptr;
    int* info = nullptr;
    int rc = RTE_OK, lw1 = 0, lw2 = 0;
    if (cudaMallocAsync(&Sp, bb * 8, s) != cudaSuccess || cudaMallocAsync(&R, bb * 8, s) != cudaSuccess ||
        cudaMallocAsync(&S, bb * 8, s) != cudaSuccess ||
        cudaMallocAsync(&info, sizeof(int) * 2 * (m + 1), s) != cudaSuccess)
        rc = fail(RTE_ERR_NOMEM, "coarse factorisation scratch");
    if (rc == RTE_OK &&
        (cusolverDnDpotrf_bufferSize(cs, CUBLAS_FILL_MODE_LOWER, Bd, S, Bd, &lw1) !=
             CUSOLVER_STATUS_SUCCESS ||
         cusolverDnDpotri_bufferSize(cs, CUBLAS_FILL_MODE_LOWER, Bd, S, Bd, &lw2) !=
             CUSOLVER_STATUS_SUCCESS))
        rc = fail(RTE_ERR_CUDA, "coarse factorisation workspace query");
    const int lw = std::max(std::max(lw1, lw2), 1);
    if (rc == RTE_OK && cudaMallocAsync(&work, sizeof(double) * lw, s) != cudaSuccess)
        rc = fail(RTE_ERR_NOMEM, "coarse factorisation workspace");
    if (rc == RTE_OK) cusolverDnSetStream(cs, s);
    const unsigned g = blocks_for(bb);
    for (int y = 0; y <= m && rc == RTE_OK; ++y) {
        if (y > 0) k_ec_schur_r<<<g, kThreads, 0, s>>>(m, dP, y, d.ec_ell, Sp, R);
        k_ec_schur_s<<<g, kThreads, 0, s>>>(m, dP, y, d.ec_ell, R, S);
        count_launches(y > 0 ? 2 : 1);
        if (cusolverDnDpotrf(cs, CUBLAS_FILL_MODE_LOWER, Bd, S, Bd, work, lw, info + 2 * y) !=
                CUSOLVER_STATUS_SUCCESS ||
            cusolverDnDpotri(cs, CUBLAS_FILL_MODE_LOWER, Bd, S, Bd, work, lw, info + 2 * y + 1) !=
                CUSOLVER_STATUS_SUCCESS) {
            rc = fail(RTE_ERR_CUDA, "coarse factorisation (cuSOLVER) failed");
            break;
        }
        const size_t o = (size_t)y * Bd * ldf;
        k_ec_store<<<blocks_for((size_t)Bd * ldf), kThreads, 0, s>>>(
            Bd, ldf, S, Sp, out32 ? out32 + o : nullptr, out64 ? out64 + o : nullptr);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) rc = fail(RTE_ERR_CUDA, "coarse factorisation kernels");
    }
    std::vector<int> hinfo(2 * (m + 1), 0);
    if (rc == RTE_OK) {
        cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * 2 * (m + 1), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess)
            rc = fail(RTE_ERR_CUDA, "coarse factorisation synchronisation");
        for (int v : hinfo)
            if (rc == RTE_OK && v != 0) rc = fail(RTE_ERR_ARG, "coarse row Schur complement is not SPD");
    }
    if (Sp) cudaFreeAsync(Sp, s);
    if (R) cudaFreeAsync(R, s);
    if (S) cudaFreeAsync(S, s);
    if (work) cudaFreeAsync(work, s);
    if (info) cudaFreeAsync(info, s);
    return rc;
}

}  // namespace rte
