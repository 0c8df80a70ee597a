// H^2-compressed scattering matrices S^+ and S^- (Section 5.2): device
// set-up of the compressed matrices and the apply Y = X S for a block of row
// vectors.  The host plan (cluster tree, boxes, block tree, block lists) is
// built in h2_build.cpp.
//
// Every stage of the apply is one block-sparse product over 64-column
// blocks, Out[:, blk j] (+)= sum_e In[:, blk in_e] B_e, with a 64 x 64 tile
// of rows per block of threads (k_h2_bsr).  The blocks of threads are
// ordered (group of 16 output blocks) x (row tile) x (output block), so that
// the blocks running at one time share their B matrices and the input
// columns of neighbouring clusters in L2.  Coupling matrices are not stored:
// K(xi^t_nu, +-xi^c_mu) is evaluated from the clusters' normalised
// interpolation points when a tile needs it (4096 kernel values against the
// tile's 2 * 64^3 multiply-adds), so that the far field costs no HBM
// traffic beyond the coefficient vectors.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "device.h"
#include "h2.h"
#include "rte_internal.h"
#include "tcgen05.cuh"

namespace rte {

namespace {

constexpr int kRT = 64;        // rows per tile of the block-sparse product
constexpr int kGroup = 16;     // output blocks per raster group
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------ set-up
// Lagrange factor l_i(x) of the per-axis nodes nd[0..p-1] (stride 3).
__device__ __forceinline__ double lagrange1(const double* nd, int p, int i, double x) {
    double v = 1.0;
    for (int j = 0; j < p; ++j)
        if (j != i) v *= (x - nd[3 * j]) / (nd[3 * i] - nd[3 * j]);
    return v;
}

// L_nu of the cluster with per-axis nodes nd [p][3] at the point x.
__device__ __forceinline__ double lagrange3(const double* nd, int p, int nu, const double* x) {
    const int ix = nu / (p * p), iy = (nu / p) % p, iz = nu % p;
    return lagrange1(nd, p, ix, x[0]) * lagrange1(nd + 1, p, iy, x[1]) *
           lagrange1(nd + 2, p, iz, x[2]);
}

__device__ __forceinline__ double hg(double mu, double g, double c0) {
    const double t = 1.0 + g * g - 2.0 * g * mu;
    return c0 / (t * sqrt(t));
}

// Leaf bases: V_t[(i, a), nu] = sum_q w phi_a(p_q) L^t_nu(p_q) over the far
// rule of representative i (phi = 1 for S^+, psi_a for S^-).  One block per
// (leaf, representative), one thread per nu.
__global__ void k_h2_leaf(int m, int p, int k, int ld_off, int qf, const double* __restrict__ nodes,
                          const double* __restrict__ pts, const double* __restrict__ w,
                          const double* __restrict__ psi, double* __restrict__ pool,
                          long long leaf0) {
    const int t = blockIdx.x, il = blockIdx.y, nu = threadIdx.x;
    const int i = t * kH2Leaf + il;
    const double* nd = nodes + (size_t)(ld_off + t) * p * 3;
    double acc[3] = {0.0, 0.0, 0.0};
    if (nu < k) {
        for (int q = 0; q < qf; ++q) {
            const double* x = pts + ((size_t)i * qf + q) * 3;
            const double v = w[(size_t)i * qf + q] * lagrange3(nd, p, nu, x);
            if (m == 1) {
                acc[0] += v;
            } else {
                const double* ps = psi + ((size_t)i * qf + q) * 3;
                for (int a = 0; a < 3; ++a) acc[a] += v * ps[a];
            }
        }
    }
    for (int a = 0; a < m; ++a) {
        const int r = il * m + a;   // row within the leaf's m * 64 rows
        pool[(leaf0 + (long long)t * m + r / kH2B) * (kH2B * kH2B) + (size_t)(r % kH2B) * kH2B + nu] =
            acc[a];
    }
}

// Transfer matrices E_c[nu', nu] = L^parent_nu(xi^c_nu') (raw tensor points
// of the child's box).  One block per child cluster.
__global__ void k_h2_transfer(int p, int k, int first, const int* __restrict__ parent,
                              const double* __restrict__ nodes, double* __restrict__ pool,
                              long long transfer0) {
    const int c = first + blockIdx.x;
    const double* ndc = nodes + (size_t)c * p * 3;
    const double* ndp = nodes + (size_t)parent[c] * p * 3;
    double* E = pool + (transfer0 + blockIdx.x) * (kH2B * kH2B);
    for (int e = threadIdx.x; e < kH2B * kH2B; e += blockDim.x) {
        const int nup = e / kH2B, nu = e % kH2B;
        double v = 0.0;
        if (nup < k && nu < k) {
            const int ix = nup / (p * p), iy = (nup / p) % p, iz = nup % p;
            const double x[3] = {ndc[3 * ix], ndc[3 * iy + 1], ndc[3 * iz + 2]};
            v = lagrange3(ndp, p, nu, x);
        }
        E[e] = v;
    }
}

// Store one entry (row (i, a), column (j, b)) of near pair `pair` in the
// B layout of its 64 x 64 chunk: B[input][output].
__device__ __forceinline__ void near_store(double* pool, long long near0, int m, int pair, int il,
                                           int a, int jl, int b, double v) {
    const int r = il * m + a, c = jl * m + b;
    const long long mat = near0 + ((long long)pair * m + r / kH2B) * m + c / kH2B;
    pool[mat * (kH2B * kH2B) + (size_t)(c % kH2B) * kH2B + (r % kH2B)] = v;
}

// Near blocks by the far rule: 2 (fd k(p.q) +- fm k(-p.q)) summed over the
// far-rule points, fd / fm the parts that are near in this pair.  One block
// per (pair, i), one thread per j.
__global__ void k_h2_near(int m, double parity, double g, int qf, const int* __restrict__ pairs,
                          const double* __restrict__ pts, const double* __restrict__ w,
                          const double* __restrict__ psi, double* __restrict__ pool,
                          long long near0) {
    const int pair = blockIdx.x, il = blockIdx.y, jl = threadIdx.x;
    const int t = pairs[3 * pair], c = pairs[3 * pair + 1], fl = pairs[3 * pair + 2];
    const int i = t * kH2Leaf + il, j = c * kH2Leaf + jl;
    const double fd = (fl & 1) ? 1.0 : 0.0, fm = (fl & 2) ? parity : 0.0;
    const double c0 = (1.0 - g * g) / (4.0 * kPi);
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < qf; ++q) {
        const double* x = pts + ((size_t)i * qf + q) * 3;
        const double wi = w[(size_t)i * qf + q];
        double row[3] = {0.0, 0.0, 0.0};
        for (int r = 0; r < qf; ++r) {
            const double* y = pts + ((size_t)j * qf + r) * 3;
            const double mu = x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
            double kv = 0.0;
            if (fd != 0.0) kv += fd * hg(mu, g, c0);
            if (fm != 0.0) kv += fm * hg(-mu, g, c0);
            kv *= w[(size_t)j * qf + r];
            if (m == 1) {
                row[0] += kv;
            } else {
                const double* pj = psi + ((size_t)j * qf + r) * 3;
                for (int b = 0; b < 3; ++b) row[b] += kv * pj[b];
            }
        }
        if (m == 1) {
            s[0] += wi * row[0];
        } else {
            const double* pi = psi + ((size_t)i * qf + q) * 3;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) s[3 * a + b] += wi * pi[a] * row[b];
        }
    }
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) near_store(pool, near0, m, pair, il, a, jl, b, 2.0 * s[3 * a + b]);
}

__device__ double block_sum256(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) s += red[i];
    return s;
}

// The pairs the dense assembly integrates by the near rule (K_j or -K_j
// shares a vertex with K_i): the entry recomputed by that rule.  One block
// of 256 threads per pair (fix = {i, j, pair}).
__global__ void __launch_bounds__(256)
k_h2_near_fix(int m, double parity, double g, int qn, const int* __restrict__ fix,
              const int* __restrict__ pairs, const double* __restrict__ pts,
              const double* __restrict__ w, const double* __restrict__ psi,
              double* __restrict__ pool, long long near0) {
    __shared__ double red[8];
    const int i = fix[3 * blockIdx.x], j = fix[3 * blockIdx.x + 1], pair = fix[3 * blockIdx.x + 2];
    const int fl = pairs[3 * pair + 2];
    const double fd = (fl & 1) ? 1.0 : 0.0, fm = (fl & 2) ? parity : 0.0;
    const double c0 = (1.0 - g * g) / (4.0 * kPi);
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < qn; q += blockDim.x) {
        const double* x = pts + ((size_t)i * qn + q) * 3;
        const double wi = w[(size_t)i * qn + q];
        double row[3] = {0.0, 0.0, 0.0};
        for (int r = 0; r < qn; ++r) {
            const double* y = pts + ((size_t)j * qn + r) * 3;
            const double mu = x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
            double kv = 0.0;
            if (fd != 0.0) kv += fd * hg(mu, g, c0);
            if (fm != 0.0) kv += fm * hg(-mu, g, c0);
            kv *= w[(size_t)j * qn + r];
            if (m == 1) {
                row[0] += kv;
            } else {
                const double* pj = psi + ((size_t)j * qn + r) * 3;
                for (int b = 0; b < 3; ++b) row[b] += kv * pj[b];
            }
        }
        if (m == 1) {
            s[0] += wi * row[0];
        } else {
            const double* pi = psi + ((size_t)i * qn + q) * 3;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) s[3 * a + b] += wi * pi[a] * row[b];
        }
    }
    const int il = i % kH2Leaf, jl = j % kH2Leaf;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            const double v = block_sum256(s[3 * a + b], red);
            if (threadIdx.x == 0) near_store(pool, near0, m, pair, il, a, jl, b, 2.0 * v);
        }
}

__global__ void k_h2_to_f32(const double* __restrict__ x, float* __restrict__ y, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}

// ------------------------------------------------------------ apply
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ void load4(const float* p, float* v) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}
__device__ __forceinline__ void store4(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float hg_t(float mu, float g, float c0) {
    const float r = rsqrtf(1.0f + g * g - 2.0f * g * mu);
    return c0 * r * r * r;
}
__device__ __forceinline__ double hg_t(double mu, double g, double c0) {
    const double t = 1.0 + g * g - 2.0 * g * mu;
    return c0 / (t * sqrt(t));
}

// Out[r, 64 out_blk[j] + q] (+)= sum_e sum_kk In[r, 64 in_blk[e] + kk] B_e[kk][q]
// for a 64-row tile.  kMode 0: B_e = pool[mat[e]]; 1: its transpose;
// 2: the coupling matrix 2 f k(s xi^out_q . xi^in_kk) with s = mat[e] the
// part's sign and f = 1 (S^+) or s (S^-), zero outside the first k rows and
// columns.  One block of 256 threads per (row tile, output block), each
// thread a 4 x 4 piece of the 64 x 64 tile; the k sum in chunks of 256 bytes
// per row staged in shared memory.
template <typename T, int kMode, bool kAccum>
__global__ void __launch_bounds__(256)
k_h2_bsr(int rows, int rtiles, int nout, int k, int parity, const T* __restrict__ In,
         long long ldi, T* __restrict__ Out, long long ldo, const int* __restrict__ out_blk,
         const int* __restrict__ ptr, const int* __restrict__ in_blk, const int* __restrict__ mat,
         const T* __restrict__ pool, const T* __restrict__ xi, T g, T c0) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    constexpr int KC = 256 / (int)sizeof(T);   // 64 floats or 32 doubles per chunk
    constexpr int VPR = KC / VN;               // 16-byte vectors per tile row
    __shared__ __align__(16) T As[kRT][KC + VN];
    __shared__ __align__(16) T Bs[KC][kH2B + VN];
    __shared__ T xo[kH2B * 3], xin[kH2B * 3];

    const long long bid = blockIdx.x;
    const long long per = (long long)kGroup * rtiles;
    const int grp = (int)(bid / per);
    const long long rem = bid % per;
    const int rt = (int)(rem / kGroup);
    const int j = grp * kGroup + (int)(rem % kGroup);
    if (j >= nout) return;
    const int r0 = rt * kRT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int ob = out_blk[j];
    if (kMode == 2)
        for (int e = tid; e < kH2B * 3; e += 256) xo[e] = xi[(size_t)ob * kH2B * 3 + e];

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = T(0);

    for (int e = ptr[j]; e < ptr[j + 1]; ++e) {
        const int ib = in_blk[e];
        const int me = mat[e];
        if (kMode == 2) {
            __syncthreads();
            for (int x = tid; x < kH2B * 3; x += 256) xin[x] = xi[(size_t)ib * kH2B * 3 + x];
        }
        for (int kc = 0; kc < kH2B; kc += KC) {
            __syncthreads();
            // A tile: 64 rows x KC columns of In
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int idx = tid + 256 * s, row = idx / VPR, cv = idx % VPR;
                V v;
                if (r0 + row < rows)
                    v = *reinterpret_cast<const V*>(In + (size_t)(r0 + row) * ldi +
                                                    (size_t)ib * kH2B + kc + cv * VN);
                else
                    memset(&v, 0, sizeof(V));
                *reinterpret_cast<V*>(&As[row][cv * VN]) = v;
            }
            // B tile: KC rows (input index) x 64 columns (output index)
            if (kMode == 0) {
                const T* B = pool + (size_t)me * (kH2B * kH2B) + (size_t)kc * kH2B;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int idx = tid + 256 * s, br = idx / (kH2B / VN), bc = idx % (kH2B / VN);
                    *reinterpret_cast<V*>(&Bs[br][bc * VN]) =
                        *reinterpret_cast<const V*>(B + (size_t)br * kH2B + bc * VN);
                }
            } else if (kMode == 1) {
                const T* B = pool + (size_t)me * (kH2B * kH2B);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int idx = tid + 256 * s, q = idx / VPR, cv = idx % VPR;
                    const V v = *reinterpret_cast<const V*>(B + (size_t)q * kH2B + kc + cv * VN);
                    const T* pv = reinterpret_cast<const T*>(&v);
#pragma unroll
                    for (int u = 0; u < VN; ++u) Bs[cv * VN + u][q] = pv[u];
                }
            } else {
                __syncthreads();   // xin staged
                const T f = T(2) * ((parity > 0 || me > 0) ? T(1) : T(-1));
                const T sg = me > 0 ? T(1) : T(-1);
                for (int idx = tid; idx < KC * kH2B; idx += 256) {
                    const int br = idx / kH2B, q = idx % kH2B, mu = kc + br;
                    T v = T(0);
                    if (mu < k && q < k) {
                        const T d = xo[3 * q] * xin[3 * mu] + xo[3 * q + 1] * xin[3 * mu + 1] +
                                    xo[3 * q + 2] * xin[3 * mu + 2];
                        v = f * hg_t(sg * d, g, c0);
                    }
                    Bs[br][q] = v;
                }
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < KC; ++kk) {
                T a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][kk];
                load4(&Bs[kk][tx * 4], b);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[i][q] = fma_t(a[i], b[q], acc[i][q]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= rows) continue;
        T* o = Out + (size_t)r * ldo + (size_t)ob * kH2B + tx * 4;
        if (kAccum) {
            T old[4];
            load4(o, old);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] += old[q];
        }
        store4(o, acc[i]);
    }
}

// ------------------------------------------------- tensor-core apply
// The same block-sparse products on the tensor cores (tcgen05, BF16
// operands, FP32 accumulation in tensor memory) for the BF16 apply.  One
// block of 128 threads per (128-row tile, output block): warp 0 lane 0 loads
// the A tile (128 rows x 64 columns of In, one 128-byte swizzled row per
// matrix row) and the B tile (the 64 x 64 matrix, stored K-major as
// Bt[output][input]) by TMA into a 4-stage ring, warp 1 lane 0 issues four
// 128 x 64 x 16 MMAs per entry, and the four warps drain the 64 accumulator
// columns.  Every wait is bounded (tc::mbar_wait).
constexpr int kTcRows = 128;
constexpr int kTcStages = 4;
constexpr uint32_t kTcABytes = kTcRows * tc::kRowBytes;   // 16 KB
constexpr uint32_t kTcBBytes = kH2B * tc::kRowBytes;      // 8 KB

constexpr size_t tc_smem_bytes() {
    return 1024 + (size_t)kTcStages * (kTcABytes + kTcBBytes) + (2 * kTcStages + 1) * 8 + 16;
}

template <bool kAccum, typename TOut>
__global__ void __launch_bounds__(128, 1)
k_h2_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
        int rows, int rtiles, int nout, TOut* __restrict__ Out, long long ldo,
        const int* __restrict__ out_blk, const int* __restrict__ ptr,
        const int* __restrict__ in_blk, const int* __restrict__ mat) {
    using namespace tc;
    constexpr uint32_t kTmemCols = kH2B;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kTcStages * kTcABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * kTcBBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 1);

    const long long bid = blockIdx.x;
    const long long per = (long long)kGroup * rtiles;
    const int grp = (int)(bid / per);
    const long long rem = bid % per;
    const int rt = (int)(rem / kGroup);
    const int j = grp * kGroup + (int)(rem % kGroup);
    if (j >= nout) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = rt * kTcRows;
    const int e0 = ptr[j], steps = ptr[j + 1] - e0;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kTcStages),
                   done = smem_u32(bars + 2 * kTcStages);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        for (int st = 0; st < steps && ok; ++st) {
            const int s = st % kTcStages;
            const uint32_t ph = (st / kTcStages) & 1;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1)) { ok = false; break; }
            mbar_expect_tx(full0 + 8 * s, kTcABytes + kTcBBytes);
            tma_load_2d(smem_u32(sA + s * kTcABytes), &mapA, full0 + 8 * s, in_blk[e0 + st] * kH2B,
                        r0);
            tma_load_2d(smem_u32(sB + s * kTcBBytes), &mapB, full0 + 8 * s, 0, mat[e0 + st] * kH2B);
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = (1u << 4)                               // D: FP32
                               | (1u << 7) | (1u << 10)                // A, B: BF16
                               | ((uint32_t)(kH2B >> 3) << 17)         // N = 64
                               | ((uint32_t)(kTcRows >> 4) << 24);     // M = 128
        for (int st = 0; st < steps && ok; ++st) {
            const int s = st % kTcStages;
            const uint32_t ph = (st / kTcStages) & 1;
            if (!mbar_wait(full0 + 8 * s, ph)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * kTcABytes), b0 = smem_u32(sB + s * kTcBBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_issue(false, tmem, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk), idesc,
                          (st > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);
    }
    __syncwarp();
    ok = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = r0 + warp * 32 + lane;
    const int ob = out_blk[j];
    for (int c0 = 0; c0 < kH2B; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (!ok || row >= rows) continue;
        if (steps == 0)
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
        TOut* dst = Out + (size_t)row * ldo + (size_t)ob * kH2B + c0;
        if constexpr (sizeof(TOut) == 4) {
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float4 w = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                if (kAccum) {
                    const float4 o = d4[i];
                    w.x += o.x; w.y += o.y; w.z += o.z; w.w += o.w;
                }
                d4[i] = w;
            }
        } else {
            uint4* d4 = reinterpret_cast<uint4*>(dst);
            uint32_t w[8];
            if (kAccum) {
                const uint4 o0 = d4[0], o1 = d4[1];
                const uint32_t ow[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&ow[i]));
                    v[2 * i] += f.x;
                    v[2 * i + 1] += f.y;
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                w[i] = *reinterpret_cast<uint32_t*>(&hv);
            }
            d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
            d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

// Matrices of the tensor-core pool in the K-major layout Bt[output][input]
// (BF16): entry e copies FP64 pool matrix src[e], transposed when tr[e].
__global__ void k_h2_tc_copy(const double* __restrict__ pool, const long long* __restrict__ src,
                             const long long* __restrict__ dst, const unsigned char* __restrict__ tr,
                             __nv_bfloat16* __restrict__ out) {
    const long long e = blockIdx.x;
    const double* S = pool + src[e] * (kH2B * kH2B);
    __nv_bfloat16* D = out + dst[e] * (kH2B * kH2B);
    const bool t = tr[e];
    for (int x = threadIdx.x; x < kH2B * kH2B; x += blockDim.x) {
        const int r = x / kH2B, c = x % kH2B;
        D[x] = __float2bfloat16_rn((float)(t ? S[c * kH2B + r] : S[x]));
    }
}

// Coupling matrices in the K-major layout: Bt[nu][mu] = 2 f k(s xi^t_nu .
// xi^c_mu) (f = 1 for S^+, s for S^-), entry e of the coupling list, whose
// row cluster is out_of[e].
__global__ void k_h2_tc_couple(int k, int parity, double g, const double* __restrict__ xi,
                               const int* __restrict__ out_of, const int* __restrict__ in_blk,
                               const int* __restrict__ sgn, __nv_bfloat16* __restrict__ out,
                               long long first) {
    const long long e = blockIdx.x;
    const double* xo = xi + (size_t)out_of[e] * kH2B * 3;
    const double* xc = xi + (size_t)in_blk[e] * kH2B * 3;
    const double s = sgn[e] > 0 ? 1.0 : -1.0;
    const double f = 2.0 * (parity > 0 ? 1.0 : s);
    const double c0 = (1.0 - g * g) / (4.0 * kPi);
    __nv_bfloat16* D = out + (first + e) * (kH2B * kH2B);
    for (int x = threadIdx.x; x < kH2B * kH2B; x += blockDim.x) {
        const int nu = x / kH2B, mu = x % kH2B;
        double v = 0.0;
        if (nu < k && mu < k) {
            const double d = xo[3 * nu] * xc[3 * mu] + xo[3 * nu + 1] * xc[3 * mu + 1] +
                             xo[3 * nu + 2] * xc[3 * mu + 2];
            v = f * hg(s * d, g, c0);
        }
        D[x] = __float2bfloat16_rn((float)v);
    }
}

struct DevList {
    int nout = 0, nnz = 0;
    int *out_blk = nullptr, *ptr = nullptr, *in_blk = nullptr, *mat = nullptr;
};

struct H2Parity {
    bool on = false;
    int m = 1;
    H2Pool pool;
    double* pool64 = nullptr;
    float* pool32 = nullptr;
    DevList up_leaf, couple, down_leaf, near;
    std::vector<DevList> up, down;
    // tensor-core (BF16) apply: matrices in the K-major layout and the same
    // lists with matrix indices into that pool
    __nv_bfloat16* tcpool = nullptr;
    long long tc_total = 0;
    DevList tc_up_leaf, tc_couple, tc_down_leaf, tc_near;
    std::vector<DevList> tc_up, tc_down;
};

int run_tc(cudaStream_t s, const DevList& L, int rows, const void* In, long long ldi,
           const __nv_bfloat16* tcpool, long long tc_total, void* Out, long long ldo, bool out_f32,
           bool accum) {
    if (L.nout == 0 || rows == 0) return RTE_OK;
    CUtensorMap ma, mb;
    RTE_TRY(tc::make_map(&ma, In, false, rows, (int)ldi, kTcRows));
    RTE_TRY(tc::make_map(&mb, tcpool, false, (int)(tc_total * kH2B), kH2B, kH2B));
    const int rtiles = (rows + kTcRows - 1) / kTcRows;
    const long long grid = (long long)((L.nout + kGroup - 1) / kGroup) * kGroup * rtiles;
    if (grid > 0x7fffffffLL) return fail(RTE_ERR_ARG, "H2 apply: too many rows for one launch");
    const size_t sm = tc_smem_bytes();
    static const bool attr = [sm] {
        cudaFuncSetAttribute(k_h2_tc<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_h2_tc<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_h2_tc<false, __nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_h2_tc<true, __nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return true;
    }();
    (void)attr;
    if (out_f32) {
        float* o = static_cast<float*>(Out);
        if (accum)
            k_h2_tc<true, float><<<(unsigned)grid, 128, sm, s>>>(ma, mb, rows, rtiles, L.nout, o, ldo,
                                                                 L.out_blk, L.ptr, L.in_blk, L.mat);
        else
            k_h2_tc<false, float><<<(unsigned)grid, 128, sm, s>>>(ma, mb, rows, rtiles, L.nout, o, ldo,
                                                                  L.out_blk, L.ptr, L.in_blk, L.mat);
    } else {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(Out);
        if (accum)
            k_h2_tc<true, __nv_bfloat16><<<(unsigned)grid, 128, sm, s>>>(
                ma, mb, rows, rtiles, L.nout, o, ldo, L.out_blk, L.ptr, L.in_blk, L.mat);
        else
            k_h2_tc<false, __nv_bfloat16><<<(unsigned)grid, 128, sm, s>>>(
                ma, mb, rows, rtiles, L.nout, o, ldo, L.out_blk, L.ptr, L.in_blk, L.mat);
    }
    count_launches(1);
    return RTE_OK;
}

template <typename T, int kMode, bool kAccum>
int run_list(cudaStream_t s, const DevList& L, int rows, int k, int parity, const T* In,
             long long ldi, T* Out, long long ldo, const T* pool, const T* xi, double g) {
    if (L.nout == 0 || rows == 0) return RTE_OK;
    const int rtiles = (rows + kRT - 1) / kRT;
    const long long grid = (long long)((L.nout + kGroup - 1) / kGroup) * kGroup * rtiles;
    if (grid > 0x7fffffffLL) return fail(RTE_ERR_ARG, "H2 apply: too many rows for one launch");
    const T c0 = T((1.0 - g * g) / (4.0 * kPi));
    k_h2_bsr<T, kMode, kAccum><<<(unsigned)grid, 256, 0, s>>>(
        rows, rtiles, L.nout, k, parity, In, ldi, Out, ldo, L.out_blk, L.ptr, L.in_blk, L.mat, pool,
        xi, T(g), c0);
    count_launches(1);
    return RTE_OK;
}

}  // namespace

}  // namespace rte

struct rte_h2 {
    rte::H2Plan plan;
    double g = 0.0;
    int precisions = 0;
    rte::H2Parity par[2];   // [0] S^+, [1] S^-
    double* xi64 = nullptr;
    float* xi32 = nullptr;
    // quadrature kept for rte_h2_dense (levels <= 5)
    double *qf_pts = nullptr, *qf_w = nullptr, *qf_psi = nullptr;
    double *qn_pts = nullptr, *qn_w = nullptr, *qn_psi = nullptr;
    int *near_ptr = nullptr, *near_idx = nullptr;
    int qf = 0, qn = 0;
    void* work = nullptr;
    size_t work_bytes = 0;
    size_t bytes = 0;
    double setup_ms = 0.0;
    std::vector<void*> allocs;
};

namespace {

template <typename T>
T* dalloc(rte_h2* h, size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) return nullptr;
    h->allocs.push_back(p);
    h->bytes += n * sizeof(T);
    return static_cast<T*>(p);
}

template <typename T>
T* upload(rte_h2* h, const std::vector<T>& v, cudaStream_t s) {
    T* d = dalloc<T>(h, v.size());
    if (d && !v.empty()) cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    return d;
}

void release(rte_h2* h, void* p) {
    for (auto& a : h->allocs)
        if (a == p) {
            cudaFree(a);
            a = nullptr;
        }
}

int upload_list(rte_h2* h, const rte::H2List& l, rte::DevList& d, cudaStream_t s) {
    d.nout = (int)l.out_blk.size();
    d.nnz = (int)l.in_blk.size();
    d.out_blk = upload(h, l.out_blk, s);
    d.ptr = upload(h, l.ptr, s);
    d.in_blk = upload(h, l.in_blk, s);
    d.mat = upload(h, l.mat, s);
    if (!d.out_blk || !d.ptr || !d.in_blk || !d.mat)
        return rte::fail(RTE_ERR_NOMEM, "H2 block lists");
    return RTE_OK;
}

}  // namespace

namespace {

template <typename T>
int h2_apply_t(rte_h2* h, int q, const T* X, T* Y, int rows, T* Xh, T* Yh, cudaStream_t s) {
    using namespace rte;
    const H2Plan& P = h->plan;
    const H2Parity& hp = h->par[q];
    const T* pool;
    const T* xi;
    if constexpr (sizeof(T) == 8) {
        pool = hp.pool64;
        xi = h->xi64;
    } else {
        pool = hp.pool32;
        xi = h->xi32;
    }
    const int parity = q == 0 ? 1 : -1;
    const long long ldx = (long long)P.n * hp.m, ldh = (long long)P.ncl * kH2B;
    const double g = h->g;
    // forward transform: leaves, then upward transfers
    RTE_TRY((run_list<T, 0, false>(s, hp.up_leaf, rows, P.k, parity, X, ldx, Xh, ldh, pool, xi, g)));
    for (int d = P.ld - 1; d >= P.dmin; --d)
        RTE_TRY((run_list<T, 0, false>(s, hp.up[d - P.dmin], rows, P.k, parity, Xh, ldh, Xh, ldh,
                                       pool, xi, g)));
    // couplings into the zeroed coefficients of the output
    cudaMemsetAsync(Yh, 0, (size_t)rows * ldh * sizeof(T), s);
    RTE_TRY((run_list<T, 2, false>(s, hp.couple, rows, P.k, parity, Xh, ldh, Yh, ldh, pool, xi, g)));
    // backward transform: downward transfers, then leaves
    for (int d = P.dmin; d < P.ld; ++d)
        RTE_TRY((run_list<T, 1, true>(s, hp.down[d - P.dmin], rows, P.k, parity, Yh, ldh, Yh, ldh,
                                      pool, xi, g)));
    RTE_TRY((run_list<T, 1, false>(s, hp.down_leaf, rows, P.k, parity, Yh, ldh, Y, ldx, pool, xi, g)));
    // near field
    RTE_TRY((run_list<T, 0, true>(s, hp.near, rows, P.k, parity, X, ldx, Y, ldx, pool, xi, g)));
    return RTE_OK;
}

}  // namespace

namespace {

// Tensor-core pool of one parity (K-major Bt[output][input] matrices, BF16):
// [leaf V^T | leaf V | E^T | E | couplings | near blocks^T] and the lists
// with matrix indices into it.
int build_tc(rte_h2* h, int q, const rte::H2Lists& lists, cudaStream_t s) {
    using namespace rte;
    const H2Plan& P = h->plan;
    H2Parity& hp = h->par[q];
    const H2Pool& pl = hp.pool;
    const long long Lc = pl.transfer0 - pl.leaf0, T = pl.near0 - pl.transfer0,
                    N = pl.total - pl.near0, F = (long long)lists.couple.in_blk.size();
    const long long Vt0 = 0, V0 = Lc, Et0 = 2 * Lc, E0 = 2 * Lc + T, C0 = 2 * Lc + 2 * T,
                    N0 = C0 + F;
    hp.tc_total = N0 + N;
    hp.tcpool = dalloc<__nv_bfloat16>(h, (size_t)hp.tc_total * kH2B * kH2B);
    if (!hp.tcpool) return fail(RTE_ERR_NOMEM, "H2 tensor-core matrices");
    std::vector<long long> src, dst;
    std::vector<unsigned char> tr;
    auto add = [&](long long a, long long b, bool t) {
        src.push_back(a);
        dst.push_back(b);
        tr.push_back(t ? 1 : 0);
    };
    for (long long i = 0; i < Lc; ++i) {
        add(pl.leaf0 + i, Vt0 + i, true);
        add(pl.leaf0 + i, V0 + i, false);
    }
    for (long long i = 0; i < T; ++i) {
        add(pl.transfer0 + i, Et0 + i, true);
        add(pl.transfer0 + i, E0 + i, false);
    }
    for (long long i = 0; i < N; ++i) add(pl.near0 + i, N0 + i, true);
    std::vector<int> out_of(F);
    for (size_t r = 0; r + 1 < lists.couple.ptr.size(); ++r)
        for (int e = lists.couple.ptr[r]; e < lists.couple.ptr[r + 1]; ++e)
            out_of[e] = lists.couple.out_blk[r];
    long long* dsrc = upload(h, src, s);
    long long* ddst = upload(h, dst, s);
    unsigned char* dtr = upload(h, tr, s);
    int* dout = upload(h, out_of, s);
    if (!dsrc || !ddst || !dtr || !dout) return fail(RTE_ERR_NOMEM, "H2 tensor-core set-up");
    if (!src.empty()) k_h2_tc_copy<<<(unsigned)src.size(), 256, 0, s>>>(hp.pool64, dsrc, ddst, dtr,
                                                                        hp.tcpool);
    if (F > 0)
        k_h2_tc_couple<<<(unsigned)F, 256, 0, s>>>(P.k, q == 0 ? 1 : -1, h->g, h->xi64, dout,
                                                   hp.couple.in_blk, hp.couple.mat, hp.tcpool, C0);
    count_launches((src.empty() ? 0 : 1) + (F > 0 ? 1 : 0));
    // the lists with tensor-core matrix indices
    auto remap = [&](const H2List& l, long long base, long long from, DevList& d) {
        H2List c = l;
        for (size_t e = 0; e < c.mat.size(); ++e)
            c.mat[e] = (int)(base + (from < 0 ? (long long)e : c.mat[e] - from));
        return upload_list(h, c, d, s);
    };
    RTE_TRY(remap(lists.up_leaf, Vt0, pl.leaf0, hp.tc_up_leaf));
    RTE_TRY(remap(lists.down_leaf, V0, pl.leaf0, hp.tc_down_leaf));
    RTE_TRY(remap(lists.couple, C0, -1, hp.tc_couple));
    RTE_TRY(remap(lists.near, N0, pl.near0, hp.tc_near));
    hp.tc_up.resize(lists.up.size());
    hp.tc_down.resize(lists.down.size());
    for (size_t d = 0; d < lists.up.size(); ++d) {
        RTE_TRY(remap(lists.up[d], Et0, pl.transfer0, hp.tc_up[d]));
        RTE_TRY(remap(lists.down[d], E0, pl.transfer0, hp.tc_down[d]));
    }
    return RTE_OK;
}

}  // namespace

namespace rte {
int h2_set_wait_cycles(long long cycles) {
    RTE_CUDA_TRY(cudaMemcpyToSymbol(tc::g_tc_wait_cycles, &cycles, sizeof(cycles)));
    return RTE_OK;
}
}  // namespace rte

extern "C" {

int rte_h2_default_options(rte_h2_options* o) {
    if (!o) return rte::fail(RTE_ERR_ARG, "options pointer is NULL");
    o->levels = 4;
    o->g = 0.5;
    o->eta = 1.4;
    o->p = 4;
    o->parities = 3;
    o->precisions = 7;
    return RTE_OK;
}

int rte_h2_create(const rte_h2_options* o, void* stream, rte_h2** out) {
    using namespace rte;
    if (!o || !out) return fail(RTE_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (o->levels < 3 || o->levels > 8)
        return fail(RTE_ERR_ARG, "H2: levels must be in [3, 8] (leaves of 64 representatives)");
    if (!(o->g >= 0.0 && o->g < 1.0)) return fail(RTE_ERR_ARG, "H2: g must satisfy 0 <= g < 1");
    if (!(o->eta > 0.0 && o->eta < 1e6)) return fail(RTE_ERR_ARG, "H2: eta must be positive");
    if (o->p < 2 || o->p > 4) return fail(RTE_ERR_ARG, "H2: p must be in [2, 4]");
    if (o->parities < 1 || o->parities > 3) return fail(RTE_ERR_ARG, "H2: parities must be 1, 2 or 3");
    if (o->precisions < 1 || o->precisions > 7)
        return fail(RTE_ERR_ARG, "H2: precisions must be a mask of 1 (FP64), 2 (FP32), 4 (BF16)");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // host: sphere, quadrature at the far and near rules, near pairs
    const SphereMesh S = make_sphere(o->levels);
    const int n = S.n;
    const int qf = 1 << (2 * kRFar), qn = 1 << (2 * kRNear);
    std::vector<double> fp((size_t)n * qf * 3), fw((size_t)n * qf), fpsi((size_t)n * qf * 3);
    std::vector<double> np((size_t)n * qn * 3), nw((size_t)n * qn), npsi((size_t)n * qn * 3);
    for (int t = 0; t < n; ++t) {
        const double* a = &S.verts[3 * S.tri[3 * t]];
        const double* b = &S.verts[3 * S.tri[3 * t + 1]];
        const double* c = &S.verts[3 * S.tri[3 * t + 2]];
        int cnt = 0;
        quad_one(a, b, c, kRFar, &fp[(size_t)t * qf * 3], &fw[(size_t)t * qf], cnt);
        cnt = 0;
        quad_one(a, b, c, kRNear, &np[(size_t)t * qn * 3], &nw[(size_t)t * qn], cnt);
        const double V[9] = {a[0], b[0], c[0], a[1], b[1], c[1], a[2], b[2], c[2]};
        double Vi[9];
        if (!inv3(V, Vi)) return fail(RTE_ERR_ARG, "degenerate sphere triangle");
        for (int rule = 0; rule < 2; ++rule) {
            const int nq = rule ? qn : qf;
            const double* P = rule ? &np[(size_t)t * qn * 3] : &fp[(size_t)t * qf * 3];
            double* Psi = rule ? &npsi[(size_t)t * qn * 3] : &fpsi[(size_t)t * qf * 3];
            for (int q = 0; q < nq; ++q)
                for (int i = 0; i < 3; ++i)
                    Psi[3 * q + i] = Vi[3 * i] * P[3 * q] + Vi[3 * i + 1] * P[3 * q + 1] +
                                     Vi[3 * i + 2] * P[3 * q + 2];
        }
    }
    std::vector<int> nptr, nidx;
    sphere_near_pairs(S, nptr, nidx);

    rte_h2* h = new rte_h2();
    H2Plan& P = h->plan;
    if (!h2_plan(o->levels, o->eta, o->p, fp, qf, P)) {
        delete h;
        return fail(RTE_ERR_ARG, "H2: degenerate cluster box");
    }
    h->g = o->g;
    h->precisions = o->precisions;
    h->qf = qf;
    h->qn = qn;
    const bool f64 = o->precisions & 1, f32 = o->precisions & 2, tcb = o->precisions & 4;

    // pools and lists per parity; memory check before any allocation
    H2Lists lists[2];
    size_t need = (size_t)n * (qf + qn) * 7 * sizeof(double) + (size_t)P.ncl * kH2B * 3 * 12;
    for (int q = 0; q < 2; ++q) {
        H2Parity& hp = h->par[q];
        hp.on = o->parities & (1 << q);
        if (!hp.on) continue;
        hp.m = q == 0 ? 1 : 3;
        hp.pool = h2_pool(P, hp.m);
        h2_lists(P, hp.pool, lists[q]);
        need += (size_t)hp.pool.total * kH2B * kH2B * (8 + (f32 ? 4 : 0));
        if (tcb)
            need += (size_t)(2 * hp.pool.total + lists[q].couple.in_blk.size()) * kH2B * kH2B * 2;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete h;
        return fail(RTE_ERR_CUDA, "cudaMemGetInfo failed");
    }
    if (need > free_b / 10 * 9) {
        delete h;
        return fail(RTE_ERR_NOMEM, "H2 matrices do not fit in free device memory");
    }

    int rc = RTE_OK;
    h->qf_pts = upload(h, fp, s);
    h->qf_w = upload(h, fw, s);
    h->qf_psi = upload(h, fpsi, s);
    h->qn_pts = upload(h, np, s);
    h->qn_w = upload(h, nw, s);
    h->qn_psi = upload(h, npsi, s);
    h->near_ptr = upload(h, nptr, s);
    h->near_idx = upload(h, nidx, s);
    double* nodes = upload(h, P.nodes, s);
    std::vector<int> parent(P.ncl, -1);
    for (int d = P.dmin + 1; d <= P.ld; ++d)
        for (int c = 0; c < P.count(d); ++c) parent[P.id(d, c)] = P.id(d - 1, c / 4);
    int* dparent = upload(h, parent, s);
    h->xi64 = upload(h, P.xi, s);
    std::vector<float> xi32(P.xi.begin(), P.xi.end());
    h->xi32 = upload(h, xi32, s);
    std::vector<int> pairs, fix;
    for (int i = 0; i < (int)P.nearm.size(); ++i) {
        const auto& pr = P.nearm[i];
        pairs.insert(pairs.end(), {pr.t, pr.c, pr.flags});
        for (int il = 0; il < kH2Leaf; ++il) {
            const int r = pr.t * kH2Leaf + il;
            for (int e = nptr[r]; e < nptr[r + 1]; ++e)
                if (nidx[e] / kH2Leaf == pr.c) fix.insert(fix.end(), {r, nidx[e], i});
        }
    }
    int* dpairs = upload(h, pairs, s);
    int* dfix = upload(h, fix, s);
    if (!h->qf_pts || !h->qf_w || !h->qf_psi || !h->qn_pts || !h->qn_w || !h->qn_psi ||
        !h->near_ptr || !h->near_idx || !nodes || !dparent || !h->xi64 || !h->xi32 || !dpairs ||
        !dfix)
        rc = fail(RTE_ERR_NOMEM, "H2 set-up arrays");

    for (int q = 0; q < 2 && rc == RTE_OK; ++q) {
        H2Parity& hp = h->par[q];
        if (!hp.on) continue;
        const double parity = q == 0 ? 1.0 : -1.0;
        const size_t elems = (size_t)hp.pool.total * kH2B * kH2B;
        hp.pool64 = dalloc<double>(h, elems);
        if (f32) hp.pool32 = dalloc<float>(h, elems);
        if (!hp.pool64 || (f32 && !hp.pool32)) {
            rc = fail(RTE_ERR_NOMEM, "H2 matrices");
            break;
        }
        cudaMemsetAsync(hp.pool64, 0, elems * sizeof(double), s);
        k_h2_leaf<<<dim3(P.leaves(), kH2Leaf), kH2B, 0, s>>>(hp.m, P.p, P.k, P.id(P.ld, 0), qf, nodes,
                                                             h->qf_pts, h->qf_w, h->qf_psi,
                                                             hp.pool64, hp.pool.leaf0);
        const int ntr = P.ncl - P.count(P.dmin);
        if (ntr > 0)
            k_h2_transfer<<<ntr, 256, 0, s>>>(P.p, P.k, P.count(P.dmin), dparent, nodes, hp.pool64,
                                              hp.pool.transfer0);
        if (!P.nearm.empty())
            k_h2_near<<<dim3((unsigned)P.nearm.size(), kH2Leaf), kH2Leaf, 0, s>>>(
                hp.m, parity, h->g, qf, dpairs, h->qf_pts, h->qf_w, h->qf_psi, hp.pool64,
                hp.pool.near0);
        if (!fix.empty())
            k_h2_near_fix<<<(unsigned)(fix.size() / 3), 256, 0, s>>>(
                hp.m, parity, h->g, qn, dfix, dpairs, h->qn_pts, h->qn_w, h->qn_psi, hp.pool64,
                hp.pool.near0);
        count_launches(2 + (ntr > 0) + !P.nearm.empty() + !fix.empty());
        if (f32) {
            k_h2_to_f32<<<(unsigned)std::min<size_t>((elems + 255) / 256, 65535u * 16u), 256, 0, s>>>(
                hp.pool64, hp.pool32, elems);
            count_launches(1);
        }
        rc = upload_list(h, lists[q].up_leaf, hp.up_leaf, s);
        if (rc == RTE_OK) rc = upload_list(h, lists[q].couple, hp.couple, s);
        if (rc == RTE_OK) rc = upload_list(h, lists[q].down_leaf, hp.down_leaf, s);
        if (rc == RTE_OK) rc = upload_list(h, lists[q].near, hp.near, s);
        hp.up.resize(lists[q].up.size());
        hp.down.resize(lists[q].down.size());
        for (size_t d = 0; d < lists[q].up.size() && rc == RTE_OK; ++d) {
            rc = upload_list(h, lists[q].up[d], hp.up[d], s);
            if (rc == RTE_OK) rc = upload_list(h, lists[q].down[d], hp.down[d], s);
        }
        if (rc == RTE_OK && tcb) rc = build_tc(h, q, lists[q], s);
    }
    if (rc == RTE_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(RTE_ERR_CUDA, std::string("H2 set-up: ") + cudaGetErrorString(e));
    }
    if (rc == RTE_OK && cudaGetLastError() != cudaSuccess) rc = fail(RTE_ERR_CUDA, "H2 set-up kernels");
    if (rc != RTE_OK) {
        rte_h2_destroy(h);
        return rc;
    }
    // set-up-only arrays
    release(h, dpairs);
    release(h, dfix);
    release(h, dparent);
    release(h, nodes);
    if (!f64)
        for (int q = 0; q < 2; ++q)
            if (h->par[q].pool64) {
                release(h, h->par[q].pool64);
                h->bytes -= (size_t)h->par[q].pool.total * kH2B * kH2B * sizeof(double);
                h->par[q].pool64 = nullptr;
            }
    if (o->levels > 5) {
        for (void* p : {(void*)h->qf_pts, (void*)h->qf_w, (void*)h->qf_psi, (void*)h->qn_pts,
                        (void*)h->qn_w, (void*)h->qn_psi, (void*)h->near_ptr, (void*)h->near_idx})
            release(h, p);
        h->qf_pts = h->qf_w = h->qf_psi = h->qn_pts = h->qn_w = h->qn_psi = nullptr;
        h->near_ptr = h->near_idx = nullptr;
    }
    h->setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return RTE_OK;
}


int rte_h2_apply(rte_h2* h, int parity, int precision, const double* X, double* Y, int rows,
                 void* stream) {
    using namespace rte;
    if (!h) return fail(RTE_ERR_ARG, "NULL handle");
    if (parity != 1 && parity != -1) return fail(RTE_ERR_ARG, "H2 apply: parity must be +1 or -1");
    const int q = parity > 0 ? 0 : 1;
    if (!h->par[q].on) return fail(RTE_ERR_ARG, "H2 apply: this parity was not built");
    if (precision != RTE_FP64 && precision != RTE_MIXED_FP32 && precision != RTE_MIXED_BF16)
        return fail(RTE_ERR_ARG, "H2 apply: precision must be RTE_FP64, RTE_MIXED_FP32 or RTE_MIXED_BF16");
    const bool fp64 = precision == RTE_FP64, bf16 = precision == RTE_MIXED_BF16;
    const int bit = fp64 ? 1 : (bf16 ? 4 : 2);
    if (!(h->precisions & bit)) return fail(RTE_ERR_ARG, "H2 apply: this precision was not built");
    if (rows < 0) return fail(RTE_ERR_ARG, "H2 apply: rows must be >= 0");
    if (rows == 0) return RTE_OK;
    if (!X || !Y) return fail(RTE_ERR_ARG, "H2 apply: NULL array");
    if (((uintptr_t)X | (uintptr_t)Y) & 15)
        return fail(RTE_ERR_ARG, "H2 apply: X and Y must be 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const H2Plan& P = h->plan;
    const size_t ncols = (size_t)P.n * h->par[q].m, nh = (size_t)P.ncl * kH2B;
    const size_t w = fp64 ? 8 : (bf16 ? 2 : 4);
    size_t need = 2 * (size_t)rows * nh * w + 1024;
    if (!fp64) need += (size_t)rows * ncols * (bf16 ? 2 : 4) + (size_t)rows * ncols * 4;
    if (need > h->work_bytes) {
        if (h->work) {
            cudaStreamSynchronize(s);
            cudaFree(h->work);
            h->work = nullptr;
            h->work_bytes = 0;
        }
        if (cudaMalloc(&h->work, need) != cudaSuccess) {
            h->work = nullptr;
            return fail(RTE_ERR_NOMEM, "H2 apply work buffers");
        }
        h->work_bytes = need;
    }
    char* wb = static_cast<char*>(h->work);
    if (bf16) {
        const H2Parity& hp = h->par[q];
        __nv_bfloat16* Xh = reinterpret_cast<__nv_bfloat16*>(wb);
        __nv_bfloat16* Yh = Xh + (size_t)rows * nh;
        __nv_bfloat16* Xb = Yh + (size_t)rows * nh;
        float* Y32 = reinterpret_cast<float*>(
            wb + ((2 * (size_t)rows * nh + (size_t)rows * ncols) * 2 + 255) / 256 * 256);
        const long long ldx = (long long)ncols, ldh = (long long)nh;
        convert(s, X, Xb, (size_t)rows * ncols);
        RTE_TRY(run_tc(s, hp.tc_up_leaf, rows, Xb, ldx, hp.tcpool, hp.tc_total, Xh, ldh, false, false));
        for (int d = P.ld - 1; d >= P.dmin; --d)
            RTE_TRY(run_tc(s, hp.tc_up[d - P.dmin], rows, Xh, ldh, hp.tcpool, hp.tc_total, Xh, ldh,
                           false, false));
        cudaMemsetAsync(Yh, 0, (size_t)rows * nh * 2, s);
        RTE_TRY(run_tc(s, hp.tc_couple, rows, Xh, ldh, hp.tcpool, hp.tc_total, Yh, ldh, false, false));
        for (int d = P.dmin; d < P.ld; ++d)
            RTE_TRY(run_tc(s, hp.tc_down[d - P.dmin], rows, Yh, ldh, hp.tcpool, hp.tc_total, Yh, ldh,
                           false, true));
        RTE_TRY(run_tc(s, hp.tc_down_leaf, rows, Yh, ldh, hp.tcpool, hp.tc_total, Y32, ldx, true,
                       false));
        RTE_TRY(run_tc(s, hp.tc_near, rows, Xb, ldx, hp.tcpool, hp.tc_total, Y32, ldx, true, true));
        convert(s, Y32, Y, (size_t)rows * ncols);
        // the pipelines' bounded waits: read the timeout flag (synchronises)
        int flag = 0;
        RTE_CUDA_TRY(cudaMemcpyFromSymbolAsync(&flag, tc::g_tc_error, sizeof(int), 0,
                                               cudaMemcpyDeviceToHost, s));
        RTE_CUDA_TRY(cudaStreamSynchronize(s));
        if (flag) {
            const int zero = 0;
            cudaMemcpyToSymbolAsync(tc::g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
            return fail(RTE_ERR_TIMEOUT, "H2 apply: a tensor-core pipeline wait timed out");
        }
    } else if (fp64) {
        double* Xh = reinterpret_cast<double*>(wb);
        double* Yh = Xh + (size_t)rows * nh;
        RTE_TRY(h2_apply_t<double>(h, q, X, Y, rows, Xh, Yh, s));
    } else {
        float* Xh = reinterpret_cast<float*>(wb);
        float* Yh = Xh + (size_t)rows * nh;
        float* X32 = Yh + (size_t)rows * nh;
        float* Y32 = X32 + (size_t)rows * ncols;
        convert(s, X, X32, (size_t)rows * ncols);
        RTE_TRY(h2_apply_t<float>(h, q, X32, Y32, rows, Xh, Yh, s));
        convert(s, Y32, Y, (size_t)rows * ncols);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RTE_ERR_CUDA, std::string("H2 apply: ") + cudaGetErrorString(e));
    return RTE_OK;
}

int rte_h2_plan_info(const rte_h2_options* o, rte_h2_info* info) {
    using namespace rte;
    if (!o || !info) return fail(RTE_ERR_ARG, "NULL argument");
    if (o->levels < 3 || o->levels > 8)
        return fail(RTE_ERR_ARG, "H2: levels must be in [3, 8] (leaves of 64 representatives)");
    if (!(o->eta > 0.0 && o->eta < 1e6)) return fail(RTE_ERR_ARG, "H2: eta must be positive");
    if (o->p < 2 || o->p > 4) return fail(RTE_ERR_ARG, "H2: p must be in [2, 4]");
    const SphereMesh S = make_sphere(o->levels);
    const int qf = 1 << (2 * kRFar);
    std::vector<double> fp((size_t)S.n * qf * 3), fw((size_t)S.n * qf);
    for (int t = 0; t < S.n; ++t) {
        int cnt = 0;
        quad_one(&S.verts[3 * S.tri[3 * t]], &S.verts[3 * S.tri[3 * t + 1]],
                 &S.verts[3 * S.tri[3 * t + 2]], kRFar, &fp[(size_t)t * qf * 3],
                 &fw[(size_t)t * qf], cnt);
    }
    H2Plan P;
    if (!h2_plan(o->levels, o->eta, o->p, fp, qf, P)) return fail(RTE_ERR_ARG, "H2: degenerate cluster box");
    std::memset(info, 0, sizeof(*info));
    info->n_plus = P.n;
    info->leaves = P.leaves();
    info->clusters = P.ncl;
    for (const auto& b : P.far) info->far_blocks[b.sign > 0 ? 0 : 1]++;
    for (const auto& b : P.near) info->near_blocks[b.sign > 0 ? 0 : 1]++;
    info->near_matrices = (int)P.nearm.size();
    info->transfers = P.ncl - P.count(P.dmin);
    return RTE_OK;
}

int rte_h2_get_info(const rte_h2* h, rte_h2_info* info) {
    using namespace rte;
    if (!h || !info) return fail(RTE_ERR_ARG, "NULL argument");
    const H2Plan& P = h->plan;
    std::memset(info, 0, sizeof(*info));
    info->n_plus = P.n;
    info->leaves = P.leaves();
    info->clusters = P.ncl;
    for (const auto& b : P.far) info->far_blocks[b.sign > 0 ? 0 : 1]++;
    for (const auto& b : P.near) info->near_blocks[b.sign > 0 ? 0 : 1]++;
    info->near_matrices = (int)P.nearm.size();
    info->transfers = P.ncl - P.count(P.dmin);
    size_t bytes = (size_t)P.ncl * kH2B * 3 * 12;
    for (int q = 0; q < 2; ++q) {
        const H2Parity& hp = h->par[q];
        if (!hp.on) continue;
        const size_t elems = (size_t)hp.pool.total * kH2B * kH2B;
        if (hp.pool64) bytes += elems * 8;
        if (hp.pool32) bytes += elems * 4;
        for (const DevList* l : {&hp.up_leaf, &hp.couple, &hp.down_leaf, &hp.near})
            bytes += sizeof(int) * (2 * (size_t)l->nout + 1 + 2 * (size_t)l->nnz);
        for (const auto& v : {&hp.up, &hp.down})
            for (const auto& l : *v) bytes += sizeof(int) * (2 * (size_t)l.nout + 1 + 2 * (size_t)l.nnz);
    }
    info->bytes = bytes;
    info->setup_ms = h->setup_ms;
    return RTE_OK;
}

int rte_h2_dense(const rte_h2* h, int parity, double* host_out, size_t n) {
    using namespace rte;
    if (!h || !host_out) return fail(RTE_ERR_ARG, "NULL argument");
    if (parity != 1 && parity != -1) return fail(RTE_ERR_ARG, "parity must be +1 or -1");
    if (!h->qf_pts) return fail(RTE_ERR_ARG, "H2 dense: only for levels <= 5");
    const int ns = h->plan.n;
    const size_t np = (size_t)ns * ns;
    if (n != (parity > 0 ? np : 9 * np)) return fail(RTE_ERR_ARG, "H2 dense: wrong output size");
    double *Sp = nullptr, *Sm = nullptr;
    if (cudaMalloc(&Sp, np * 8) != cudaSuccess) return fail(RTE_ERR_NOMEM, "H2 dense");
    if (cudaMalloc(&Sm, 9 * np * 8) != cudaSuccess) {
        cudaFree(Sp);
        return fail(RTE_ERR_NOMEM, "H2 dense");
    }
    QuadDev qd{h->qn_pts, h->qn_w, h->qn_psi, h->qf_pts, h->qf_w, h->qf_psi,
               h->near_ptr, h->near_idx, h->qn, h->qf};
    cudaStream_t s = nullptr;
    assemble_scattering(s, ns, h->g, qd, Sp, Sm);
    cudaMemcpyAsync(host_out, parity > 0 ? Sp : Sm, n * 8, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(Sp);
    cudaFree(Sm);
    if (e != cudaSuccess) return fail(RTE_ERR_CUDA, std::string("H2 dense: ") + cudaGetErrorString(e));
    return RTE_OK;
}

void rte_h2_destroy(rte_h2* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    if (h->work) cudaFree(h->work);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
