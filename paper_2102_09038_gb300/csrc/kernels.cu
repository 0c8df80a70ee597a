// FP64 CUDA kernels of the hot path: Kronecker-structured transport and
// mass applies (eq. AR, bMebMo with eq. tpmv), the scattering and eigenbasis
// contractions (eq. bKebKo, Lemma apply_high_order_pre), the coarse-matrix
// apply, per-RHS reductions, and the setup-time quadrature of S^+ / S^-.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "device.h"
#include "rte_internal.h"

namespace rte {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(size_t n, int threads = kThreads) {
    size_t b = (n + threads - 1) / threads;
    const size_t cap = 65535ull * 32ull;
    return (unsigned)std::max<size_t>(1, std::min(b, cap));
}

// ------------------------------------------------------------------ GEMM
// Row-major C = alpha * (A B) .* F + beta * C, 64 x 64 tiles, 16-deep K
// steps, 256 threads with a 4 x 4 register tile each.
template <int EPI>
__global__ void __launch_bounds__(256)
k_gemm_f64(int M, int N, int K, const double* __restrict__ A, int lda,
           const double* __restrict__ B, int ldb, double* C, int ldc,
           double alpha, double beta, const double* __restrict__ at,
           const double* __restrict__ as, const double* __restrict__ lam,
           int rows) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 2];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = threadIdx.x + t * 256;
            const int r = e >> 4, c = e & 15;
            const int gr = m0 + r, gc = k0 + c;
            As[c][r] = (gr < M && gc < K) ? A[(size_t)gr * lda + gc] : 0.0;
            const int br = e >> 6, bc = e & 63;
            const int gbr = k0 + br, gbc = n0 + bc;
            Bs[br][bc] = (gbr < K && gbc < N) ? B[(size_t)gbr * ldb + gbc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = m0 + ty + 16 * i;
        if (r >= M) continue;
        double fat = 0.0, fas = 0.0;
        if (EPI != 0) {
            const int rr = r % rows;
            fat = at[rr];
            fas = as[rr];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx + 16 * j;
            if (c >= N) continue;
            double v = acc[i][j];
            if (EPI == 1) v = v / (fat - lam[c] * fas);
            if (EPI == 2) v = v * (1.0 / (fat - lam[c] * fas) - 1.0 / fat);
            v *= alpha;
            double* dst = C + (size_t)r * ldc + c;
            if (beta != 0.0) v += beta * *dst;
            *dst = v;
        }
    }
}

// ----------------------------------------------------- transport A (a1)
// Z[r, j, 3k+c] = sum_n A_n(k, c) (D_n U_r)[j, k]; computed in TC, read as TIn,
// written as TOut (FP64, or FP32 in / BF16-or-FP32 out for the mixed paths)
template <typename TIn, typename TOut, typename TC>
__global__ void k_apply_A(int nRm, int nRp, int nSp, int nrhs,
                          const int* __restrict__ cell_nodes,
                          const TC* __restrict__ cell_D,
                          const TC* __restrict__ A1,
                          const TC* __restrict__ A2,
                          const TIn* __restrict__ U, TOut* __restrict__ Z) {
    const unsigned total = (unsigned)nrhs * nRm * nSp;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int k = (int)(e % (unsigned)nSp);
        const unsigned rj = e / (unsigned)nSp;
        const int j = (int)(rj % (unsigned)nRm);
        const int r = (int)(rj / (unsigned)nRm);
        const TIn* Ur = U + (size_t)r * nRp * nSp;
        TC g1 = 0, g2 = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const TC u = static_cast<TC>(Ur[(size_t)cell_nodes[3 * j + a] * nSp + k]);
            g1 = fma(cell_D[6 * j + a], u, g1);
            g2 = fma(cell_D[6 * j + 3 + a], u, g2);
        }
        TOut* z = Z + rj * (3 * (size_t)nSp) + 3 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c) z[c] = static_cast<TOut>(A1[3 * k + c] * g1 + A2[3 * k + c] * g2);
    }
}

// ------------------------------------------ A^T + M^+ + R - K^+ (a2, b2)
template <typename T>
__global__ void k_apply_even(int nRm, int nRp, int nSp, int nrhs, int nnz,
                             int flags, const int* __restrict__ adj_ptr,
                             const int* __restrict__ adj_cell,
                             const int* __restrict__ adj_loc,
                             const T* __restrict__ cell_D,
                             const T* __restrict__ A1,
                             const T* __restrict__ A2,
                             const int* __restrict__ st_ptr,
                             const int* __restrict__ st_col,
                             const T* __restrict__ sval,
                             const T* __restrict__ m,
                             const T* __restrict__ omx,
                             const T* __restrict__ omy,
                             const T* __restrict__ Zp,
                             const T* __restrict__ X,
                             const T* __restrict__ V, T* __restrict__ Y) {
    const unsigned total = (unsigned)nrhs * nRp * nSp;
    const T* Mt = sval + (size_t)kMt * nnz;
    const T* Ms = sval + (size_t)kMs * nnz;
    const T* Bx = sval + (size_t)kBx * nnz;
    const T* By = sval + (size_t)kBy * nnz;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int k = (int)(e % (unsigned)nSp);
        const unsigned ri = e / (unsigned)nSp;
        const int i = (int)(ri % (unsigned)nRp);
        const int r = (int)(ri / (unsigned)nRp);
        T acc = 0;
        if (flags & 1) {
            const T a1[3] = {A1[3 * k], A1[3 * k + 1], A1[3 * k + 2]};
            const T a2[3] = {A2[3 * k], A2[3 * k + 1], A2[3 * k + 2]};
            const T* Zr = Zp + (size_t)r * nRm * 3 * nSp;
            for (int p = adj_ptr[i]; p < adj_ptr[i + 1]; ++p) {
                const int j = adj_cell[p], a = adj_loc[p];
                const T* z = Zr + (size_t)j * 3 * nSp + 3 * k;
                const T t1 = a1[0] * z[0] + a1[1] * z[1] + a1[2] * z[2];
                const T t2 = a2[0] * z[0] + a2[1] * z[1] + a2[2] * z[2];
                acc += cell_D[6 * j + a] * t1 + cell_D[6 * j + 3 + a] * t2;
            }
        }
        if (flags & 6) {
            const T mk = m[k], ox = omx[k], oy = omy[k];
            const T* Xr = X + (size_t)r * nRp * nSp;
            const T* Vr = V ? V + (size_t)r * nRp * nSp : nullptr;
            for (int p = st_ptr[i]; p < st_ptr[i + 1]; ++p) {
                const size_t col = (size_t)st_col[p] * nSp + k;
                if (flags & 2) acc += (mk * Mt[p] + ox * Bx[p] + oy * By[p]) * Xr[col];
                if (flags & 4) acc -= Ms[p] * Vr[col];
            }
        }
        Y[e] = acc;
    }
}

// (M^- - K^-) z = at_j (z_j M_S^-) - as_j (z_j S^-),  G = Z S^- precomputed
__global__ void k_mk_combine(int nRm, int nSp, int nrhs,
                             const double* __restrict__ at,
                             const double* __restrict__ as,
                             const double* __restrict__ MSm,
                             const double* __restrict__ Z,
                             const double* __restrict__ G, double* __restrict__ Y) {
    const unsigned total = (unsigned)nrhs * nRm * nSp;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int k = (int)(e % (unsigned)nSp);
        const unsigned rj = e / (unsigned)nSp;
        const int j = (int)(rj % (unsigned)nRm);
        const size_t base = rj * 3 * nSp + 3 * k;
        const double z[3] = {Z[base], Z[base + 1], Z[base + 2]};
        const double* M = MSm + 9 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double mz = M[3 * c] * z[0] + M[3 * c + 1] * z[1] + M[3 * c + 2] * z[2];
            Y[base + c] = at[j] * mz - as[j] * G[base + c];
        }
    }
}

// Y = (B M_S^{-1}) / at   (the high-order part of eq. MmKprecond)
__global__ void k_mk_minv_scale(int nRm, int nSp, int nrhs,
                                const double* __restrict__ at,
                                const double* __restrict__ MSm_inv,
                                const double* __restrict__ B, double* __restrict__ Y) {
    const unsigned total = (unsigned)nrhs * nRm * nSp;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int k = (int)(e % (unsigned)nSp);
        const unsigned rj = e / (unsigned)nSp;
        const int j = (int)(rj % (unsigned)nRm);
        const size_t base = rj * 3 * nSp + 3 * k;
        const double b[3] = {B[base], B[base + 1], B[base + 2]};
        const double* M = MSm_inv + 9 * k;
        const double inv = 1.0 / at[j];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Y[base + c] = (M[3 * c] * b[0] + M[3 * c + 1] * b[1] + M[3 * c + 2] * b[2]) * inv;
    }
}

__global__ void k_rhs_source(int nRp, int nSp, int nrhs, int nnz,
                             const int* __restrict__ st_ptr,
                             const int* __restrict__ st_col,
                             const double* __restrict__ sval,
                             const double* __restrict__ m,
                             const double* __restrict__ qn, double* __restrict__ q) {
    const size_t total = (size_t)nrhs * nRp * nSp;
    const double* Mu = sval + (size_t)kMu * nnz;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % nSp);
        const size_t ri = e / nSp;
        const int i = (int)(ri % nRp);
        const int r = (int)(ri / nRp);
        double s = 0.0;
        for (int p = st_ptr[i]; p < st_ptr[i + 1]; ++p)
            s += Mu[p] * qn[(size_t)r * nRp + st_col[p]];
        q[e] = s * m[k];
    }
}

// Inflow part of l^+ (Section 2.4): 2 (|s.n| g, phi_i mu_k) over the
// incoming half of the boundary.  On face f with outward normal n, exactly
// one triangle of pair k has s.n < 0 (the octahedral sphere mesh has no
// triangle across a coordinate plane): half[f][k] says which.  Its integral
// of |s.n| is half of omega_k (omega^x on the faces x = 0, 1, omega^y on
// y = 0, 1), and the data is P1 along the face, so
//   q[i(f, j)][k] += omega_k sum_j' B1[j][j'] g[f][j'][2k + half[f][k]]
// with B1 the face's 1-D P1 mass (h/3 at the ends, 2h/3 inside, h/6 off the
// diagonal, h = 1/m).  One launch takes the two opposite faces f0, f0 + 1,
// whose nodes are disjoint, so no two threads add to one entry.
__global__ void k_inflow(int m, int nSp, int nrhs, int f0, const int* __restrict__ half,
                         const double* __restrict__ omx, const double* __restrict__ omy,
                         const double* __restrict__ g, double* __restrict__ q) {
    const int nf = m + 1, nRp = nf * nf;
    const size_t total = (size_t)nrhs * 2 * nf * nSp;
    const double h = 1.0 / m;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % nSp);
        size_t rest = e / nSp;
        const int j = (int)(rest % nf);
        rest /= nf;
        const int f = f0 + (int)(rest % 2);
        const int r = (int)(rest / 2);
        const int hk = half[f * nSp + k];
        const double* gf = g + ((size_t)r * 4 + f) * nf * 2 * nSp + 2 * k + hk;
        const double gj = gf[(size_t)j * 2 * nSp];
        double acc = (j == 0 || j == m ? h / 3.0 : 2.0 * h / 3.0) * gj;
        if (j > 0) acc += h / 6.0 * gf[(size_t)(j - 1) * 2 * nSp];
        if (j < m) acc += h / 6.0 * gf[(size_t)(j + 1) * 2 * nSp];
        const double om = f < 2 ? omx[k] : omy[k];
        // node of face f's j-th point: x = 0 / x = 1 run along y, y = 0 / y = 1 along x
        const int i = f == 0 ? j * nf : f == 1 ? j * nf + m : f == 2 ? j : m * nf + j;
        q[((size_t)r * nRp + i) * nSp + k] += om * acc;
    }
}

// ------------------------------------------------------------ reductions
template <int BS>
__device__ double block_sum(double v) {
    __shared__ double sh[BS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < BS / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// x[e] uniform in [-1, 1) from the SplitMix64 mix of (seed, e) (Steele,
// Lea and Flood, "Fast splittable pseudorandom number generators", 2014).
__global__ void k_fill_uniform(double* __restrict__ x, size_t n, unsigned long long seed) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (e + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[e] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_dot_partial(const T* __restrict__ x, const T* __restrict__ y,
              size_t len, double* __restrict__ partial) {
    const int r = blockIdx.y;
    const T* xr = x + (size_t)r * len;
    const T* yr = y + (size_t)r * len;
    double s = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len;
         e += (size_t)gridDim.x * blockDim.x)
        s = fma((double)xr[e], (double)yr[e], s);
    s = block_sum<256>(s);
    if (threadIdx.x == 0) partial[(size_t)r * 1024 + blockIdx.x] = s;
}

__global__ void __launch_bounds__(256)
k_dot_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    const int r = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(size_t)r * 1024 + b];
    s = block_sum<256>(s);
    if (threadIdx.x == 0) out[r] = s;
}

template <typename T>
__global__ void k_axpby(const T* __restrict__ x, T* __restrict__ y,
                        size_t len, int nrhs, const double* __restrict__ a,
                        double ca, const double* __restrict__ b, double cb) {
    const unsigned total = (unsigned)(len * nrhs);
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int r = nrhs == 1 ? 0 : (int)(e / (unsigned)len);
        const T av = static_cast<T>(a ? a[r] : ca);
        const T bv = static_cast<T>(b ? b[r] : cb);
        const T yv = bv == T(0) ? T(0) : bv * y[e];
        y[e] = (x ? av * x[e] : T(0)) + yv;
    }
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ x, TO* __restrict__ y, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        y[e] = static_cast<TO>(x[e]);
}

// --------------------------------------------------------- coarse apply
// Y[r, i, a] = sum_p sum_b Ec[p, a, b] X[r, col(p), b]
__global__ void k_coarse_apply(int nRp, int d, int nrhs, const int* __restrict__ st_ptr,
                               const int* __restrict__ st_col,
                               const double* __restrict__ ec,
                               const double* __restrict__ X, double* __restrict__ Y) {
    const size_t total = (size_t)nrhs * nRp * d;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % d);
        const size_t ri = e / d;
        const int i = (int)(ri % nRp);
        const int r = (int)(ri / nRp);
        const double* Xr = X + (size_t)r * nRp * d;
        double s = 0.0;
        for (int p = st_ptr[i]; p < st_ptr[i + 1]; ++p) {
            const double* blk = ec + ((size_t)p * d + a) * d;
            const double* xv = Xr + (size_t)st_col[p] * d;
            for (int b = 0; b < d; ++b) s = fma(blk[b], xv[b], s);
        }
        Y[e] = s;
    }
}

// ------------------------------------------------ quadrature of S^+, S^-
__device__ __forceinline__ double hg_eval(double mu, double g, double c0) {
    const double t = 1.0 + g * g - 2.0 * g * mu;
    return c0 / (t * sqrt(t));
}

// Far rule for every pair: one thread per (k, k').
__global__ void k_scatter_far(int n, double g, const double* __restrict__ pts,
                              const double* __restrict__ w,
                              const double* __restrict__ psi, int qf,
                              double* __restrict__ Sp, double* __restrict__ Sm) {
    const size_t pair = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (pair >= (size_t)n * n) return;
    const int k = (int)(pair / n), kk = (int)(pair % n);
    const double c0 = (1.0 - g * g) / (4.0 * 3.14159265358979323846);
    double sp = 0.0, sm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = 0; p < qf; ++p) {
        const double* s = pts + ((size_t)k * qf + p) * 3;
        const double wp = w[(size_t)k * qf + p];
        const double* ps = psi + ((size_t)k * qf + p) * 3;
        double rowp = 0.0, rowm[3] = {0, 0, 0};
        for (int q = 0; q < qf; ++q) {
            const double* t = pts + ((size_t)kk * qf + q) * 3;
            const double mu = s[0] * t[0] + s[1] * t[1] + s[2] * t[2];
            const double kp = hg_eval(mu, g, c0), km = hg_eval(-mu, g, c0);
            const double wq = w[(size_t)kk * qf + q];
            const double* pq = psi + ((size_t)kk * qf + q) * 3;
            rowp += wq * (kp + km);
            const double dk = wq * (kp - km);
            rowm[0] += dk * pq[0];
            rowm[1] += dk * pq[1];
            rowm[2] += dk * pq[2];
        }
        sp += wp * rowp;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) sm[3 * i + j] += wp * ps[i] * rowm[j];
    }
    Sp[(size_t)k * n + kk] = 2.0 * sp;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Sm[(size_t)(3 * k + i) * 3 * n + 3 * kk + j] = 2.0 * sm[3 * i + j];
}

// Near rule for vertex-sharing pairs: one block per (k, k'), one thread per
// node of K_k.
__global__ void __launch_bounds__(256)
k_scatter_near(int n, double g, const double* __restrict__ pts,
               const double* __restrict__ w, const double* __restrict__ psi, int qn,
               const int* __restrict__ near_ptr, const int* __restrict__ near_idx,
               const int* __restrict__ pair_row, double* __restrict__ Sp,
               double* __restrict__ Sm) {
    const int pidx = blockIdx.x;
    const int k = pair_row[pidx];
    const int kk = near_idx[pidx];
    const double c0 = (1.0 - g * g) / (4.0 * 3.14159265358979323846);
    double sp = 0.0, sm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < qn; p += blockDim.x) {
        const double* s = pts + ((size_t)k * qn + p) * 3;
        const double wp = w[(size_t)k * qn + p];
        const double* ps = psi + ((size_t)k * qn + p) * 3;
        double rowp = 0.0, rowm[3] = {0, 0, 0};
        for (int q = 0; q < qn; ++q) {
            const double* t = pts + ((size_t)kk * qn + q) * 3;
            const double mu = s[0] * t[0] + s[1] * t[1] + s[2] * t[2];
            const double kp = hg_eval(mu, g, c0), km = hg_eval(-mu, g, c0);
            const double wq = w[(size_t)kk * qn + q];
            const double* pq = psi + ((size_t)kk * qn + q) * 3;
            rowp += wq * (kp + km);
            const double dk = wq * (kp - km);
            rowm[0] += dk * pq[0];
            rowm[1] += dk * pq[1];
            rowm[2] += dk * pq[2];
        }
        sp += wp * rowp;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) sm[3 * i + j] += wp * ps[i] * rowm[j];
    }
    sp = block_sum<256>(sp);
    if (threadIdx.x == 0) Sp[(size_t)k * n + kk] = 2.0 * sp;
    for (int c = 0; c < 9; ++c) {
        const double v = block_sum<256>(sm[c]);
        if (threadIdx.x == 0)
            Sm[(size_t)(3 * k + c / 3) * 3 * n + 3 * kk + c % 3] = 2.0 * v;
    }
}

__global__ void k_symmetrise(int n, double* __restrict__ S) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e >= (size_t)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    if (j <= i) return;
    const double v = 0.5 * (S[(size_t)i * n + j] + S[(size_t)j * n + i]);
    S[(size_t)i * n + j] = v;
    S[(size_t)j * n + i] = v;
}

__global__ void k_e0_coef(int nRp, int nSp, const double* __restrict__ ell6,
                          const double* __restrict__ e0s, double* __restrict__ coef,
                          float* __restrict__ coef_f) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t per = (size_t)7 * nRp;
    if (e >= per * nSp) return;
    const size_t di = e / nSp;          // dir * nRp + i
    const int k = (int)(e % nSp);
    double c = 0.0;
    for (int q = 0; q < 6; ++q) c += e0s[6 * k + q] * ell6[(size_t)q * per + di];
    coef[e] = c;
    if (coef_f) coef_f[e] = (float)c;
}

__global__ void k_near_rows(int n, const int* __restrict__ near_ptr, int* __restrict__ row) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    for (int p = near_ptr[k]; p < near_ptr[k + 1]; ++p) row[p] = k;
}

// ------------------------------------------- structured-mesh versions
// The m x m "/"-mesh: node (x, y) = y (m+1) + x; square (I, J) holds cells
// 2 (J m + I) (lower: (I,J),(I+1,J),(I+1,J+1)) and 2 (J m + I) + 1 (upper:
// (I,J),(I+1,J+1),(I,J+1)).  Adjacency is computed, not looked up.
template <typename TIn, typename TOut, typename TC>
__global__ void k_apply_A_s(int m, int nSp, int nrhs, const TC* __restrict__ cell_D,
                            const TC* __restrict__ A1, const TC* __restrict__ A2,
                            const TIn* __restrict__ U, TOut* __restrict__ Z) {
    const int nRm = 2 * m * m, nRp = (m + 1) * (m + 1);
    const unsigned total = (unsigned)nrhs * nRm * nSp;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int k = (int)(e % (unsigned)nSp);
        const unsigned rj = e / (unsigned)nSp;
        const int j = (int)(rj % (unsigned)nRm);
        const int r = (int)(rj / (unsigned)nRm);
        const int q = j >> 1, I = q % m, J = q / m;
        const int n00 = J * (m + 1) + I;
        const int nd[3] = {n00, (j & 1) ? n00 + m + 2 : n00 + 1,
                           (j & 1) ? n00 + m + 1 : n00 + m + 2};
        const TIn* Ur = U + (size_t)r * nRp * nSp + k;
        TC g1 = 0, g2 = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const TC u = static_cast<TC>(Ur[(size_t)nd[a] * nSp]);
            g1 = fma(cell_D[6 * j + a], u, g1);
            g2 = fma(cell_D[6 * j + 3 + a], u, g2);
        }
        TOut* z = Z + (size_t)rj * (3 * (size_t)nSp) + 3 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            z[c] = static_cast<TOut>(A1[3 * k + c] * g1 + A2[3 * k + c] * g2);
    }
}

// Y = [A^T Zp] + [M^+ X + R X] - [M_s^+ V] on the structured mesh; ell4 holds
// M_t^+, M_s^+, B_x, B_y in ELL form [4][7][nRp].
template <typename T>
__global__ void k_apply_even_s(int m, int nSp, int nrhs, int flags,
                               const T* __restrict__ cell_D, const T* __restrict__ A1,
                               const T* __restrict__ A2, const T* __restrict__ ell4,
                               const T* __restrict__ mk, const T* __restrict__ omx,
                               const T* __restrict__ omy, const T* __restrict__ Zp,
                               const T* __restrict__ X, const T* __restrict__ V,
                               T* __restrict__ Y) {
    const int nRp = (m + 1) * (m + 1), nRm = 2 * m * m;
    const unsigned total = (unsigned)nrhs * nRp * nSp;
    const int off[7] = {0, 1, -1, m + 1, -(m + 1), m + 2, -(m + 2)};
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int k = (int)(e % (unsigned)nSp);
        const unsigned ri = e / (unsigned)nSp;
        const int i = (int)(ri % (unsigned)nRp);
        const int r = (int)(ri / (unsigned)nRp);
        const int x = i % (m + 1), y = i / (m + 1);
        T acc = 0;
        if (flags & 1) {
            const T a1[3] = {A1[3 * k], A1[3 * k + 1], A1[3 * k + 2]};
            const T a2[3] = {A2[3 * k], A2[3 * k + 1], A2[3 * k + 2]};
            const T* Zr = Zp + (size_t)r * nRm * 3 * nSp + 3 * k;
            // the six cells around node (x, y) and the node's local index
            const int cI[6] = {x, x, x - 1, x - 1, x - 1, x};
            const int cJ[6] = {y, y, y, y - 1, y - 1, y - 1};
            const int up[6] = {0, 1, 0, 0, 1, 1};
            const int loc[6] = {0, 0, 1, 2, 1, 2};
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                if (cI[t] < 0 || cJ[t] < 0 || cI[t] >= m || cJ[t] >= m) continue;
                const int j = 2 * (cJ[t] * m + cI[t]) + up[t];
                const T* z = Zr + (size_t)j * 3 * nSp;
                const T z0 = z[0], z1 = z[1], z2 = z[2];
                const T t1 = a1[0] * z0 + a1[1] * z1 + a1[2] * z2;
                const T t2 = a2[0] * z0 + a2[1] * z1 + a2[2] * z2;
                acc += cell_D[6 * j + loc[t]] * t1 + cell_D[6 * j + 3 + loc[t]] * t2;
            }
        }
        if (flags & 6) {
            const T mkv = mk[k], ox = omx[k], oy = omy[k];
            const T* Xr = X + (size_t)r * nRp * nSp + k;
            const T* Vr = V ? V + (size_t)r * nRp * nSp + k : nullptr;
            const size_t sl = (size_t)7 * nRp;
#pragma unroll
            for (int dir = 0; dir < 7; ++dir) {
                int jn = i + off[dir];
                jn = jn < 0 ? 0 : (jn >= nRp ? nRp - 1 : jn);
                const size_t pe = (size_t)dir * nRp + i;
                if (flags & 2)
                    acc += (mkv * ell4[pe] + ox * ell4[2 * sl + pe] + oy * ell4[3 * sl + pe]) *
                           Xr[(size_t)jn * nSp];
                if (flags & 4) acc -= ell4[sl + pe] * Vr[(size_t)jn * nSp];
            }
        }
        Y[e] = acc;
    }
}

}  // namespace

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

void gemm_f64(cudaStream_t s, int M, int N, int K, const double* A, int lda,
              const double* B, int ldb, double* C, int ldc, double alpha,
              double beta, int epi, const double* at, const double* as,
              const double* lam, int rows) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    count_launches(1);
    if (epi == 1)
        k_gemm_f64<1><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, at, as, lam, rows);
    else if (epi == 2)
        k_gemm_f64<2><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, at, as, lam, rows);
    else
        k_gemm_f64<0><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, at, as, lam, rows);
}

void apply_A(cudaStream_t s, const DevSystem& d, const double* U, double* Z, int nrhs) {
    const size_t total = (size_t)nrhs * d.nRm * d.nSp;
    count_launches(1);
    k_apply_A_s<double, double, double><<<grid_for(total, d.tpb_A), d.tpb_A, 0, s>>>(
        d.m, d.nSp, nrhs, d.cell_D, d.ang_A1, d.ang_A2, U, Z);
}

void apply_A_lo(cudaStream_t s, const DevSystem& d, const float* U, void* Z, bool bf16,
                int nrhs) {
    const size_t total = (size_t)nrhs * d.nRm * d.nSp;
    count_launches(1);
    if (bf16)
        k_apply_A_s<float, __nv_bfloat16, float><<<grid_for(total, d.tpb_A), d.tpb_A, 0, s>>>(
            d.m, d.nSp, nrhs, d.lo.cell_D, d.lo.A1, d.lo.A2, U, static_cast<__nv_bfloat16*>(Z));
    else
        k_apply_A_s<float, float, float><<<grid_for(total, d.tpb_A), d.tpb_A, 0, s>>>(
            d.m, d.nSp, nrhs, d.lo.cell_D, d.lo.A1, d.lo.A2, U, static_cast<float*>(Z));
}

void apply_even(cudaStream_t s, const DevSystem& d, const double* Zp, const double* X,
                const double* V, double* Y, int nrhs, int flags) {
    const size_t total = (size_t)nrhs * d.nRp * d.nSp;
    count_launches(1);
    k_apply_even_s<double><<<grid_for(total, d.tpb_even), d.tpb_even, 0, s>>>(
        d.m, d.nSp, nrhs, flags, d.cell_D, d.ang_A1, d.ang_A2, d.ell4, d.ang_m, d.ang_omx,
        d.ang_omy, Zp, X, V, Y);
}

void apply_even_lo(cudaStream_t s, const DevSystem& d, const float* Zp, const float* X,
                   const float* V, float* Y, int nrhs, int flags) {
    const size_t total = (size_t)nrhs * d.nRp * d.nSp;
    count_launches(1);
    k_apply_even_s<float><<<grid_for(total, d.tpb_even), d.tpb_even, 0, s>>>(
        d.m, d.nSp, nrhs, flags, d.lo.cell_D, d.lo.A1, d.lo.A2, d.lo.ell4, d.lo.m, d.lo.omx,
        d.lo.omy, Zp, X, V, Y);
}

void mk_combine(cudaStream_t s, const DevSystem& d, const double* Z, const double* G,
                double* Y, int nrhs) {
    const size_t total = (size_t)nrhs * d.nRm * d.nSp;
    count_launches(1);
    k_mk_combine<<<grid_for(total), kThreads, 0, s>>>(d.nRm, d.nSp, nrhs, d.cell_at,
                                                      d.cell_as, d.ang_MSm, Z, G, Y);
}

void mk_minv_scale(cudaStream_t s, const DevSystem& d, const double* B, double* Y,
                   int nrhs) {
    const size_t total = (size_t)nrhs * d.nRm * d.nSp;
    count_launches(1);
    k_mk_minv_scale<<<grid_for(total), kThreads, 0, s>>>(d.nRm, d.nSp, nrhs, d.cell_at,
                                                         d.ang_MSm_inv, B, Y);
}

void inflow_source(cudaStream_t s, const DevSystem& d, const double* g, double* q, int nrhs) {
    const size_t total = (size_t)nrhs * 2 * (d.m + 1) * d.nSp;
    for (int f0 = 0; f0 < 4; f0 += 2)
        k_inflow<<<grid_for(total), kThreads, 0, s>>>(d.m, d.nSp, nrhs, f0, d.inflow_half,
                                                     d.ang_omx, d.ang_omy, g, q);
    count_launches(2);
}

void rhs_source(cudaStream_t s, const DevSystem& d, const double* qn, double* q, int nrhs) {
    const size_t total = (size_t)nrhs * d.nRp * d.nSp;
    count_launches(1);
    k_rhs_source<<<grid_for(total), kThreads, 0, s>>>(d.nRp, d.nSp, nrhs, d.nnz, d.st_ptr,
                                                      d.st_col, d.sval, d.ang_m, qn, q);
}

template <typename T>
void dot_impl(cudaStream_t s, const T* x, const T* y, size_t len, int nrhs, double* partial,
              double* out) {
    int nb = (int)std::min<size_t>(1024, std::max<size_t>(1, (len + 2047) / 2048));
    count_launches(2);
    k_dot_partial<T><<<dim3(nb, nrhs), 256, 0, s>>>(x, y, len, partial);
    k_dot_final<<<nrhs, 256, 0, s>>>(partial, nb, out);
}

void dot_per_rhs(cudaStream_t s, const double* x, const double* y, size_t len, int nrhs,
                 double* partial, double* out) {
    dot_impl(s, x, y, len, nrhs, partial, out);
}

void dot_per_rhs(cudaStream_t s, const float* x, const float* y, size_t len, int nrhs,
                 double* partial, double* out) {
    dot_impl(s, x, y, len, nrhs, partial, out);
}

void axpby_per_rhs(cudaStream_t s, const double* x, double* y, size_t len, int nrhs,
                   const double* a, double ca, const double* b, double cb) {
    count_launches(1);
    k_axpby<double><<<grid_for(len * nrhs), kThreads, 0, s>>>(x, y, len, nrhs, a, ca, b, cb);
}

void axpby_per_rhs(cudaStream_t s, const float* x, float* y, size_t len, int nrhs,
                   const double* a, double ca, const double* b, double cb) {
    count_launches(1);
    k_axpby<float><<<grid_for(len * nrhs), kThreads, 0, s>>>(x, y, len, nrhs, a, ca, b, cb);
}

void fill_uniform(cudaStream_t s, double* x, size_t n, unsigned long long seed) {
    count_launches(1);
    k_fill_uniform<<<grid_for(n), kThreads, 0, s>>>(x, n, seed);
}


// ------------------------------------------ restriction and prolongation
// qc[row][j] = sum_k x[row][k] W[k][j], one warp per row: lanes stride over
// k with 16 partial sums each, reduced across the warp by halving exchanges
// (31 shuffles leave lane j holding the sum of column j mod 16).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(int rows, int nSp, int dP, const double* __restrict__ x,
                                                  const T* __restrict__ W, double* __restrict__ qc) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= rows) return;
    T v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = T(0);
    const double* xr = x + (size_t)row * nSp;
    for (int k = lane; k < nSp; k += 32) {
        const T xv = (T)__ldg(xr + k);
        const T* w = W + (size_t)k * dP;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < dP) v[j] = fma(xv, __ldg(w + j), v[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const T send = up ? v[i] : v[i + o];
            const T keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (lane < dP) qc[(size_t)row * dP + lane] = (double)v[0];
}

// x[row][k] = beta x[row][k] + sum_j uc[row][j] WT[j][k], one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(int rows, int nSp, int dP, const double* __restrict__ uc,
                                                 const T* __restrict__ WT, double* __restrict__ x,
                                                 double beta) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= rows) return;
    const T mine = lane < dP ? (T)uc[(size_t)row * dP + lane] : T(0);
    T u[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) u[j] = __shfl_sync(0xffffffffu, mine, j);
    double* xr = x + (size_t)row * nSp;
    for (int k = lane; k < nSp; k += 32) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < dP) acc = fma(u[j], __ldg(WT + (size_t)j * nSp + k), acc);
        xr[k] = beta == 0.0 ? (double)acc : beta * xr[k] + (double)acc;
    }
}

bool restrict_rows(cudaStream_t s, int rows, int nSp, int dP, const double* x, const double* W,
                   const float* W32, double* qc) {
    if (dP < 1 || dP > 16 || rows <= 0) return false;
    const unsigned blocks = (unsigned)(((size_t)rows * 32 + 255) / 256);
    count_launches(1);
    if (W32)
        k_restrict<float><<<blocks, 256, 0, s>>>(rows, nSp, dP, x, W32, qc);
    else
        k_restrict<double><<<blocks, 256, 0, s>>>(rows, nSp, dP, x, W, qc);
    return true;
}

bool prolong_rows(cudaStream_t s, int rows, int nSp, int dP, const double* uc, const double* WT,
                  const float* WT32, double* x, double beta) {
    if (dP < 1 || dP > 16 || rows <= 0) return false;
    const unsigned blocks = (unsigned)(((size_t)rows * 32 + 255) / 256);
    count_launches(1);
    if (WT32)
        k_prolong<float><<<blocks, 256, 0, s>>>(rows, nSp, dP, uc, WT32, x, beta);
    else
        k_prolong<double><<<blocks, 256, 0, s>>>(rows, nSp, dP, uc, WT, x, beta);
    return true;
}

void convert(cudaStream_t s, const double* x, float* y, size_t n) {
    count_launches(1);
    k_convert<double, float><<<grid_for(n), kThreads, 0, s>>>(x, y, n);
}

void convert(cudaStream_t s, const float* x, double* y, size_t n) {
    count_launches(1);
    k_convert<float, double><<<grid_for(n), kThreads, 0, s>>>(x, y, n);
}

void convert(cudaStream_t s, const float* x, __nv_bfloat16* y, size_t n) {
    count_launches(1);
    k_convert<float, __nv_bfloat16><<<grid_for(n), kThreads, 0, s>>>(x, y, n);
}

void convert(cudaStream_t s, const double* x, __nv_bfloat16* y, size_t n) {
    count_launches(1);
    k_convert<double, __nv_bfloat16><<<grid_for(n), kThreads, 0, s>>>(x, y, n);
}

void coarse_apply(cudaStream_t s, const DevSystem& d, const double* X, double* Y, int nrhs) {
    const size_t total = (size_t)nrhs * d.nRp * d.dP;
    count_launches(1);
    k_coarse_apply<<<grid_for(total), kThreads, 0, s>>>(d.nRp, d.dP, nrhs, d.st_ptr,
                                                        d.st_col, d.ec_val, X, Y);
}

void e0_coefficients(cudaStream_t s, int nRp, int nSp, const double* ell6, const double* e0s,
                     double* coef, float* coef_f) {
    const size_t n = (size_t)7 * nRp * nSp;
    k_e0_coef<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nRp, nSp, ell6, e0s, coef, coef_f);
}

void assemble_scattering(cudaStream_t s, int n, double g, const QuadDev& q, double* Sp,
                         double* Sm) {
    const size_t pairs = (size_t)n * n;
    k_scatter_far<<<(unsigned)((pairs + 127) / 128), 128, 0, s>>>(
        n, g, q.far_pts, q.far_w, q.far_psi, q.qf, Sp, Sm);
    // near pairs: row index of every entry of the near list
    int npairs = 0;
    cudaMemcpyAsync(&npairs, q.near_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int* rows = nullptr;
    if (npairs > 0 && cudaMallocAsync(&rows, sizeof(int) * npairs, s) == cudaSuccess) {
        k_near_rows<<<(n + 127) / 128, 128, 0, s>>>(n, q.near_ptr, rows);
        k_scatter_near<<<npairs, 256, 0, s>>>(n, g, q.near_pts, q.near_w, q.near_psi, q.qn,
                                              q.near_ptr, q.near_idx, rows, Sp, Sm);
        cudaFreeAsync(rows, s);
    }
    k_symmetrise<<<grid_for(pairs), kThreads, 0, s>>>(n, Sp);
    const size_t pm = (size_t)9 * n * n;
    k_symmetrise<<<grid_for(pm), kThreads, 0, s>>>(3 * n, Sm);
}

}  // namespace rte
