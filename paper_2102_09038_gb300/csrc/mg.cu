// Multigrid-preconditioned conjugate gradients, each solve in one persistent
// cooperative kernel:
//  * E_0^{-1} (eq. equivalence_bE_bE0): the n_S^+ decoupled direction blocks,
//    block k = gamma (a11 K11 + a12 K12 + a22 K22) + om^x B_x + om^y B_y +
//    m_k M_t^+, all (rhs, direction) columns at once, each column stopping
//    on its own relative residual.  Multigrid is the route the paper names for
//    these anisotropic diffusion blocks (Section 5.5).
//  * E_c^{-1} (Section 5.4): the coarse Galerkin system, d x d blocks on the
//    node stencil, one CG per right-hand side.
// The preconditioner is one symmetric V-cycle in FP32 on the nested meshes:
// damped Jacobi (block Jacobi for E_c) smoothing, nu sweeps before and after,
// restriction P^T, a dense inverse on the coarsest level.  The CG recurrences
// run in the solve's precision T with FP64 reductions.  Operators are in the
// 7-direction ELL form of mg.h with computed neighbour indices; blocks meet
// at bounded grid barriers (persist.cuh).
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

__device__ __forceinline__ int nbr(int i, int dir, int m, int n) {
    const int off[7] = {0, 1, -1, m + 1, -(m + 1), m + 2, -(m + 2)};
    const int j = i + off[dir];
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

// restriction P^T: fine node q of coarse node I's list (the fine nodes that
// interpolate from I, with their weights; width Cv.rwid, zero-weight padding)
__device__ __forceinline__ int restrict_src(const MGDeviceLevel& Cv, int I, int q, float& w) {
    const size_t k = (size_t)I * Cv.rwid + q;
    w = __ldg(Cv.rw + k);
    return __ldg(Cv.ridx + k);
}

// prolongation: coarse nodes (and weights) interpolating fine node i; the
// coarse mesh is the floor(mf/2)-mesh, and for odd mf the last fine column
// and row take the values of the ones before them
__device__ __forceinline__ void prolong_src(int i, int mf, int& c0, int& c1, float& w0,
                                            float& w1) {
    const int mc = mf / 2;
    const int x = min(i % (mf + 1), 2 * mc), y = min(i / (mf + 1), 2 * mc);
    if (!(x & 1) && !(y & 1)) {
        c0 = c1 = (y / 2) * (mc + 1) + x / 2;
        w0 = 1.f;
        w1 = 0.f;
    } else if ((x & 1) && !(y & 1)) {
        c0 = (y / 2) * (mc + 1) + (x - 1) / 2;
        c1 = c0 + 1;
        w0 = w1 = 0.5f;
    } else if (!(x & 1)) {
        c0 = ((y - 1) / 2) * (mc + 1) + x / 2;
        c1 = c0 + (mc + 1);
        w0 = w1 = 0.5f;
    } else {
        c0 = ((y - 1) / 2) * (mc + 1) + (x - 1) / 2;
        c1 = c0 + (mc + 2);
        w0 = w1 = 0.5f;
    }
}

// Grid-stride loop over the items (i, c) = (e / nc, e % nc) of an n x nc
// array, with the quotient and remainder advanced incrementally (no division
// inside the loop).  Item counts stay below 2^31.
#define ITEMS(n, ncv)                                                           \
    {                                                                            \
    const unsigned it_nc__ = (unsigned)(ncv);                                    \
    const unsigned it_total__ = (unsigned)(n) * it_nc__;                         \
    const unsigned it_stride__ = gridDim.x * blockDim.x;                         \
    const unsigned it_sq__ = it_stride__ / it_nc__, it_sr__ = it_stride__ % it_nc__; \
    unsigned e = blockIdx.x * blockDim.x + threadIdx.x;                          \
    int i = (int)(e / it_nc__), c = (int)(e % it_nc__);                          \
    for (; e < it_total__; e += it_stride__, i += it_sq__, c += it_sr__,         \
                           (c >= (int)it_nc__ ? (c -= it_nc__, ++i) : 0))

// ================================================================ E_0 V-cycle
struct E0MG {
    int L, ncols, nSp, nu;
    bool dense;
    const float* cinv;     // [n_c][n_c][nSp]
    const float4* w8;      // [nSp][2]: gamma a11, gamma a12, gamma a22, om^x, om^y, m, 0, 0
    const float4* wq;      // [6][nSp / 4]: the same weights, direction index fastest
    const MGDeviceLevel* lev;   // [L], in device memory
};

// The E_0 block of direction k is sum_q w_q(k) S_q over the six spatial parts
// S_q (K11, K12, K22, B_x, B_y, M_t on level 0, their Galerkin products below),
// so its stencil coefficients are formed on the fly from the level's parts,
// stored node-major as sv[i][dir][8] (six used), and the direction's weights:
// the sweeps read 224 bytes per node instead of 28 bytes per (node,
// direction) pair.
__device__ __forceinline__ float e0_coef(const float4* sv, float4 wa, float4 wb, int i, int dir) {
    const float4 a = __ldg(sv + ((size_t)i * 7 + dir) * 2);
    const float4 b = __ldg(sv + ((size_t)i * 7 + dir) * 2 + 1);
    return fmaf(wa.x, a.x, fmaf(wa.y, a.y, fmaf(wa.z, a.z, fmaf(wa.w, a.w,
           fmaf(wb.x, b.x, wb.y * b.y)))));
}

// The V-cycle works on quads: a thread takes four consecutive columns (four
// directions) of one node, so the node's parts are read once for four
// columns and every vector access is one 16-byte load or store.  The
// columns of a level are ncols = nrhs n_S^+, a multiple of 4.
struct Quad {
    float4 w[6];   // weights of the quad's four directions, w[q].x for the first
    int k4 = -1;   // which quad of directions w holds
    __device__ void load(const float4* wq, int nq_dir, int k4new) {
        if (k4new == k4) return;
#pragma unroll
        for (int q = 0; q < 6; ++q) w[q] = __ldg(wq + (size_t)q * nq_dir + k4new);
        k4 = k4new;
    }
    // the four coefficients of stencil direction dir at node i
    __device__ __forceinline__ float4 coef(const float4* sv, int i, int dir) const {
        const float4 a = __ldg(sv + ((size_t)i * 7 + dir) * 2);
        const float2 b = __ldg(reinterpret_cast<const float2*>(sv + ((size_t)i * 7 + dir) * 2 + 1));
        float4 c;
        c.x = fmaf(w[0].x, a.x, fmaf(w[1].x, a.y, fmaf(w[2].x, a.z, fmaf(w[3].x, a.w,
              fmaf(w[4].x, b.x, w[5].x * b.y)))));
        c.y = fmaf(w[0].y, a.x, fmaf(w[1].y, a.y, fmaf(w[2].y, a.z, fmaf(w[3].y, a.w,
              fmaf(w[4].y, b.x, w[5].y * b.y)))));
        c.z = fmaf(w[0].z, a.x, fmaf(w[1].z, a.y, fmaf(w[2].z, a.z, fmaf(w[3].z, a.w,
              fmaf(w[4].z, b.x, w[5].z * b.y)))));
        c.w = fmaf(w[0].w, a.x, fmaf(w[1].w, a.y, fmaf(w[2].w, a.z, fmaf(w[3].w, a.w,
              fmaf(w[4].w, b.x, w[5].w * b.y)))));
        return c;
    }
};

__device__ __forceinline__ float4 ld4(const float4* p) { return __ldcg(p); }

// y = (E_0 block) x for the quad (i, p); dg = its diagonal
__device__ __forceinline__ float4 e0_apply4(const MGDeviceLevel& L, const Quad& qd,
                                            const float4* x4, int i, int p, int nq, float4& dg) {
    const float4* sv = reinterpret_cast<const float4*>(L.sv);
    // the seven neighbour loads first (long latency), then the coefficients
    // one direction at a time (L1 hits), to bound the live registers
    float4 xv[7];
#pragma unroll
    for (int dir = 0; dir < 7; ++dir) xv[dir] = ld4(x4 + (size_t)nbr(i, dir, L.m, L.n) * nq + p);
    float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int dir = 0; dir < 7; ++dir) {
        asm volatile("" ::: "memory");
        const float4 cf = qd.coef(sv, i, dir);
        y.x = fmaf(cf.x, xv[dir].x, y.x);
        y.y = fmaf(cf.y, xv[dir].y, y.y);
        y.z = fmaf(cf.z, xv[dir].z, y.z);
        y.w = fmaf(cf.w, xv[dir].w, y.w);
        if (dir == 0) dg = cf;
    }
    return y;
}

// The V-cycle visits only the active quads of the iteration: ql lists them
// (increasing, na of them; ql == nullptr: all nq quads).  A quad whose four
// columns have converged is left alone on every level, since nothing reads
// its values again.
__device__ __forceinline__ int quad_at(const unsigned short* ql, int k) {
    return ql ? (int)ql[k] : k;
}

// Loop over the active quads (i, p) of an n-node level with nq quads per
// node; o4 = the quad's float4 offset.  Thread t keeps active quad t % na
// for all its nodes (t / na, stepping by the grid's threads / na; the last
// threads / na * na .. threads - 1 idle), so its four directions' weights
// are loaded once.  Needs nq, nqd (direction quads), ql, na and wq in scope.
#define QUADS(n, UNROLL)                                                        \
    {                                                                            \
    const int kq__ = nqd - 1;   /* n_S^+ is a power of two */                    \
    const unsigned qd_na__ = na > 0 ? (unsigned)na : 1u;                         \
    const unsigned qd_rows__ = gridDim.x * blockDim.x / qd_na__;                 \
    const unsigned qd_t__ = blockIdx.x * blockDim.x + threadIdx.x;               \
    const bool qd_on__ = na > 0 && qd_t__ < qd_rows__ * qd_na__;                 \
    const int p = qd_on__ ? quad_at(ql, (int)(qd_t__ % qd_na__)) : 0;            \
    Quad qd;                                                                     \
    if (qd_on__) qd.load(wq, nqd, p & kq__);                                     \
    _Pragma(UNROLL)                                                              \
    for (int i = (int)(qd_t__ / qd_na__); qd_on__ && i < (int)(n);               \
         i += (int)qd_rows__) {                                                  \
        const size_t o4 = (size_t)i * nq + p;

__device__ __forceinline__ float4 jac4(float4 x, float4 b, float4 y, float4 d) {
    return make_float4(x.x + kOmega * __fdividef(b.x - y.x, d.x),
                       x.y + kOmega * __fdividef(b.y - y.y, d.y),
                       x.z + kOmega * __fdividef(b.z - y.z, d.z),
                       x.w + kOmega * __fdividef(b.w - y.w, d.w));
}

// The V-cycle's phases, each compiled on its own (not inlined) so that its
// registers are allocated for its own loop alone.
__device__ __noinline__ void e0_first(const MGDeviceLevel Lv, const float4* __restrict__ wq,
                                      int nq, int nqd, const unsigned short* __restrict__ ql,
                                      int na, float4* __restrict__ x) {
    const float4* __restrict__ B = reinterpret_cast<const float4*>(Lv.B);
    const float4* __restrict__ sv = reinterpret_cast<const float4*>(Lv.sv);
    QUADS(Lv.n, "unroll 2")
        const float4 d = qd.coef(sv, i, 0), b = ld4(B + o4);
        x[o4] = make_float4(kOmega * __fdividef(b.x, d.x), kOmega * __fdividef(b.y, d.y),
                            kOmega * __fdividef(b.z, d.z), kOmega * __fdividef(b.w, d.w));
    }}
}

__device__ __noinline__ void e0_jacobi(const MGDeviceLevel Lv, const float4* __restrict__ wq,
                                       int nq, int nqd, const unsigned short* __restrict__ ql,
                                       int na, const float4* __restrict__ x,
                                       float4* __restrict__ xt) {
    const float4* __restrict__ B = reinterpret_cast<const float4*>(Lv.B);
    QUADS(Lv.n, "unroll 2")
        float4 dg;
        const float4 y = e0_apply4(Lv, qd, x, i, p, nq, dg);
        xt[o4] = jac4(ld4(x + o4), ld4(B + o4), y, dg);
    }}
}

__device__ __noinline__ void e0_residual(const MGDeviceLevel Lv, const float4* __restrict__ wq,
                                         int nq, int nqd, const unsigned short* __restrict__ ql,
                                         int na, const float4* __restrict__ x,
                                         float4* __restrict__ t) {
    const float4* __restrict__ B = reinterpret_cast<const float4*>(Lv.B);
    QUADS(Lv.n, "unroll 2")
        float4 dg;
        const float4 y = e0_apply4(Lv, qd, x, i, p, nq, dg);
        const float4 b = ld4(B + o4);
        t[o4] = make_float4(b.x - y.x, b.y - y.y, b.z - y.z, b.w - y.w);
    }}
}

__device__ __noinline__ void e0_restrict(const MGDeviceLevel Cv, int nq,
                                         const unsigned short* __restrict__ ql, int na,
                                         const float4* __restrict__ t) {
    float4* __restrict__ CB = reinterpret_cast<float4*>(Cv.B);
    const unsigned total = (unsigned)Cv.n * (unsigned)na;
#pragma unroll 2
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int i = (int)(e / (unsigned)na), p = quad_at(ql, (int)(e % (unsigned)na));
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < Cv.rwid; ++q) {
            float w;
            const int f = restrict_src(Cv, i, q, w);
            const float4 v = ld4(t + (size_t)f * nq + p);
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
            acc.z = fmaf(w, v.z, acc.z);
            acc.w = fmaf(w, v.w, acc.w);
        }
        CB[(size_t)i * nq + p] = acc;
    }
}

__device__ __noinline__ void e0_prolong(const MGDeviceLevel Lv, int nq,
                                        const unsigned short* __restrict__ ql, int na,
                                        float4* __restrict__ x, const float4* __restrict__ xc) {
    const unsigned total = (unsigned)Lv.n * (unsigned)na;
#pragma unroll 2
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += gridDim.x * blockDim.x) {
        const int i = (int)(e / (unsigned)na), p = quad_at(ql, (int)(e % (unsigned)na));
        const size_t o4 = (size_t)i * nq + p;
        int c0, c1;
        float w0, w1;
        prolong_src(i, Lv.m, c0, c1, w0, w1);
        const float4 a = ld4(xc + (size_t)c0 * nq + p), b = ld4(xc + (size_t)c1 * nq + p);
        const float4 v = ld4(x + o4);
        x[o4] = make_float4(v.x + w0 * a.x + w1 * b.x, v.y + w0 * a.y + w1 * b.y,
                           v.z + w0 * a.z + w1 * b.z, v.w + w0 * a.w + w1 * b.w);
    }
}

// coarsest level: x = (dense inverse of each direction block) B, for the
// active quads.  cinv is [direction][i][j], rows padded with zeros to n4 (a
// multiple of 4) so that lanes read them as float4.  Work units are (active
// quad, chunk of rows), about one per block: the block stages the quad's
// four B columns in shared memory (zero past n), and each warp takes a row
// at a time with its lanes over j, for the quad's four directions: up to 12
// independent 512-byte warp loads in flight, each inverse row read once.
__device__ __noinline__ void e0_dense(const MGDeviceLevel Lv, const float* __restrict__ cinv,
                                      int nSp, int nc, const unsigned short* __restrict__ ql,
                                      int na, float* __restrict__ x) {
    constexpr int kN4 = (kDenseCoarseNodes + 3) & ~3;
    constexpr int kTrips = (kN4 / 4 + 31) / 32;
    __shared__ __align__(16) float sB[4][kN4];
    const int n = Lv.n, n4 = (n + 3) & ~3, q4 = n4 >> 2;
    const int kq = (nSp >> 2) - 1;   // n_S^+ = 4^(levels + 1)
    const int chunks = max(1, min(n, (int)gridDim.x / max(na, 1)));
    const int rows = (n + chunks - 1) / chunks;
    const int units = na * chunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int k = u / chunks, h = u - k * chunks;
        const int p = quad_at(ql, k);
        const int col0 = 4 * p, d0 = 4 * (p & kq);
        __syncthreads();   // the previous unit's reads of sB are done
        for (int t = threadIdx.x; t < 4 * n4; t += blockDim.x) {
            const int j = t >> 2;
            sB[t & 3][j] = j < n ? ldg2(Lv.B + (size_t)j * nc + col0 + (t & 3)) : 0.f;
        }
        __syncthreads();
        const int i_end = min(n, (h + 1) * rows);
        for (int i = h * rows + warp; i < i_end; i += nw) {
            float a0[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t < kTrips; ++t) {
                const int j4 = lane + 32 * t;
                if (j4 < q4) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4* r = reinterpret_cast<const float4*>(
                                              cinv + (size_t)(d0 + c) * n * n4) + j4;
                        const float4 b = reinterpret_cast<const float4*>(sB[c])[j4];
                        const float4 v = __ldg(r + (size_t)i * q4);
                        a0[c] = fmaf(v.x, b.x, fmaf(v.y, b.y, fmaf(v.z, b.z, fmaf(v.w, b.w, a0[c]))));
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a0[c] += __shfl_xor_sync(0xffffffffu, a0[c], o);
            if (lane < 4)
                x[(size_t)i * nc + col0 + lane] =
                    lane == 0 ? a0[0] : lane == 1 ? a0[1] : lane == 2 ? a0[2] : a0[3];
        }
    }
}

// One symmetric V-cycle on B_0 over the quads ql lists (na of them; all
// quads when ql is null); returns the buffer holding z on level 0.
__device__ bool e0_vcycle(const E0MG& mg, GridBar* bar, float*& z,
                          const unsigned short* ql = nullptr, int na = -1) {
    const int nc = mg.ncols, nq = nc >> 2, nqd = mg.nSp >> 2;
    if (!ql) na = nq;
    z = mg.lev[0].X;
    if (na <= 0) return true;
    int cur[kMaxMGLevels];
    for (int l = 0; l < mg.L; ++l) cur[l] = 0;
    auto buf4 = [&](int l, int which) {
        return reinterpret_cast<float4*>(which ? mg.lev[l].Xt : mg.lev[l].X);
    };
    for (int l = 0; l + 1 < mg.L; ++l) {
        const MGDeviceLevel Lv = mg.lev[l];
        e0_first(Lv, mg.wq, nq, nqd, ql, na, buf4(l, 0));
        cur[l] = 0;
        if (!grid_sync(bar)) return false;
        for (int k = 1; k < mg.nu; ++k) {
            e0_jacobi(Lv, mg.wq, nq, nqd, ql, na, buf4(l, cur[l]), buf4(l, cur[l] ^ 1));
            cur[l] ^= 1;
            if (!grid_sync(bar)) return false;
        }
        float4* t = buf4(l, cur[l] ^ 1);
        e0_residual(Lv, mg.wq, nq, nqd, ql, na, buf4(l, cur[l]), t);
        if (!grid_sync(bar)) return false;
        e0_restrict(mg.lev[l + 1], nq, ql, na, t);
        if (!grid_sync(bar)) return false;
    }
    {
        const int l = mg.L - 1;
        const MGDeviceLevel Lv = mg.lev[l];
        if (mg.dense) {
            e0_dense(Lv, mg.cinv, mg.nSp, nc, ql, na, reinterpret_cast<float*>(buf4(l, 0)));
            cur[l] = 0;
            if (!grid_sync(bar)) return false;
        } else {
            e0_first(Lv, mg.wq, nq, nqd, ql, na, buf4(l, 0));
            cur[l] = 0;
            if (!grid_sync(bar)) return false;
            for (int k = 1; k < kCoarseSweeps; ++k) {
                e0_jacobi(Lv, mg.wq, nq, nqd, ql, na, buf4(l, cur[l]), buf4(l, cur[l] ^ 1));
                cur[l] ^= 1;
                if (!grid_sync(bar)) return false;
            }
        }
    }
    for (int l = mg.L - 2; l >= 0; --l) {
        const MGDeviceLevel Lv = mg.lev[l];
        e0_prolong(Lv, nq, ql, na, buf4(l, cur[l]), buf4(l + 1, cur[l + 1]));
        if (!grid_sync(bar)) return false;
        for (int k = 0; k < mg.nu; ++k) {
            e0_jacobi(Lv, mg.wq, nq, nqd, ql, na, buf4(l, cur[l]), buf4(l, cur[l] ^ 1));
            cur[l] ^= 1;
            if (!grid_sync(bar)) return false;
        }
    }
    z = reinterpret_cast<float*>(buf4(0, cur[0]));
    return true;
}

// ================================================================ E_0 PCG
template <typename T>
struct E0Args {
    int nRp, m, nSp, nrhs, ncols, kTiles, chunks, units, maxit;
    double tol2;
    const T* coef;      // FP64: level-0 coefficients [7][nRp][nSp]; FP32: unused
    const double* B;
    double* X;
    T* R;
    T* P;
    T* AP;
    float* X32;         // FP32 kernel: the iterate (X written at the end)
    double* acc;        // [3 slots][3][ncols]: pAp, rz, rr
    double* bb;
    GridBar* bar;
    SolveStatus* status;
    E0MG mg;
};

constexpr int kChunk = 128;  // nodes per work unit (8 rows x 16 passes)

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
__global__ void __launch_bounds__(256, 2) k_e0_pcg(E0Args<T> a) {
    constexpr bool kOnTheFly = sizeof(T) == sizeof(float);
    __shared__ double sh[256];
    __shared__ int s_stop;
    const int kx = threadIdx.x & 31, ny = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_stop = 0;
    const int nc = a.ncols;
    float* B0 = a.mg.lev[0].B;
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
#define NODE_PAIR_LOOP                                              \
    for (int t = 0; t < kChunk / 16; ++t) {                         \
        const int ia = chunk * kChunk + ny + 8 * t, ib = ia + kChunk / 2; \
        if (ia >= a.nRp) break;                                     \
        const bool vb = ib < a.nRp;                                 \
        const size_t ea = ((size_t)r * a.nRp + ia) * a.nSp + k;     \
        const size_t eb = ea + (size_t)(kChunk / 2) * a.nSp;
// Four nodes per trip (i0 + 0, 32, 64, 96 of the unit's rows): every load of
// the four is issued before the first store.
#define NODE4_LOOP                                                  \
    for (int t = 0; t < kChunk / 32; ++t) {                         \
        const int i0 = chunk * kChunk + ny + 8 * t;                 \
        if (i0 >= a.nRp) break;                                     \
        int iv[4];                                                  \
        bool vv[4];                                                 \
        size_t ev[4], emv[4];                                       \
        _Pragma("unroll") for (int q = 0; q < 4; ++q) {             \
            iv[q] = i0 + q * (kChunk / 4);                          \
            vv[q] = iv[q] < a.nRp;                                  \
            ev[q] = ((size_t)r * a.nRp + iv[q]) * a.nSp + k;        \
            emv[q] = (size_t)iv[q] * nc + col;                      \
        }
    // ------------------------------------------------------------ init
    UNIT_LOOP
        double pbb = 0.0;
        if (kv) {
            NODE4_LOOP
                T bv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vv[q]) bv[q] = static_cast<T>(a.B[ev[q]]);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vv[q]) {
                        a.X[ev[q]] = 0.0;
                        a.R[ev[q]] = bv[q];
                        B0[emv[q]] = static_cast<float>(bv[q]);
                        pbb += (double)bv[q] * (double)bv[q];
                    }
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
            NODE4_LOOP
                T zv[4], rv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vv[q]) {
                        zv[q] = static_cast<T>(ldg2(z + emv[q]));
                        rv[q] = ldg2(a.R + ev[q]);
                    }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vv[q]) {
                        a.P[ev[q]] = zv[q];
                        prz += (double)rv[q] * (double)zv[q];
                    }
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
                // FP32: coefficients formed on the fly from the level-0 parts;
                // FP64: read from the precomputed FP64 stencil
                float4 wa = make_float4(0.f, 0.f, 0.f, 0.f), wb = wa;
                const float4* sv0 = reinterpret_cast<const float4*>(a.mg.lev[0].sv);
                if (kOnTheFly) {
                    wa = __ldg(a.mg.w8 + 2 * k);
                    wb = __ldg(a.mg.w8 + 2 * k + 1);
                }
                auto cf = [&](int i, int dir) -> T {
                    if (kOnTheFly) return static_cast<T>(e0_coef(sv0, wa, wb, i, dir));
                    return __ldg(a.coef + ((size_t)dir * a.nRp + i) * a.nSp + k);
                };
                // nodes ia and ib = ia + kChunk / 2 together, loads before stores
                NODE_PAIR_LOOP
                    T ya = 0, yb = 0, pb = 0;
#pragma unroll
                    for (int dir = 0; dir < 7; ++dir)
                        ya += cf(ia, dir) * ldg2(Pr + (size_t)nbr(ia, dir, a.m, a.nRp) * a.nSp + k);
                    const T pa = ldg2(a.P + ea);
                    if (vb) {
#pragma unroll
                        for (int dir = 0; dir < 7; ++dir)
                            yb += cf(ib, dir) *
                                  ldg2(Pr + (size_t)nbr(ib, dir, a.m, a.nRp) * a.nSp + k);
                        pb = ldg2(a.P + eb);
                    }
                    a.AP[ea] = ya;
                    ppap += (double)ya * (double)pa;
                    if (vb) {
                        a.AP[eb] = yb;
                        ppap += (double)yb * (double)pb;
                    }
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
                NODE4_LOOP
                    if (act) {
                        double xo[4];
                        T pv[4], rv[4], apv[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (vv[q]) {
                                xo[q] = ldg2(a.X + ev[q]);
                                pv[q] = ldg2(a.P + ev[q]);
                                rv[q] = ldg2(a.R + ev[q]);
                                apv[q] = ldg2(a.AP + ev[q]);
                            }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (vv[q]) {
                                a.X[ev[q]] = xo[q] + alpha * (double)pv[q];
                                const T rn = rv[q] - static_cast<T>(alpha) * apv[q];
                                a.R[ev[q]] = rn;
                                prr += (double)rn * (double)rn;
                                B0[emv[q]] = static_cast<float>(rn);
                            }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (vv[q]) B0[emv[q]] = 0.f;
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
            NODE4_LOOP
                T nv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vv[q])
                        nv[q] = static_cast<T>(ldg2(z + emv[q])) +
                                static_cast<T>(beta) * ldg2(a.P + ev[q]);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (vv[q]) a.P[ev[q]] = nv[q];
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
#undef NODE_PAIR_LOOP
#undef NODE4_LOOP
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status->iterations = it;
        a.status->converged = s_stop;
    }
}

__device__ __forceinline__ float4 ldf4q(const float* base, size_t o4) {
    return __ldcg(reinterpret_cast<const float4*>(base) + o4);
}

// ------------------------------------------ E_0 PCG, FP32, quad phases
// The FP32 CG runs as the V-cycle does: grid-stride loops over quads (four
// consecutive columns of one node), each phase its own function.  The CG
// vectors keep the even layout [rhs][node][direction]; the V-cycle arrays
// are [node][column].  Per-column dot products: every thread sums its
// quad's four columns over its nodes in FP32 (a few dozen products at most
// at level 0); a block combines its threads in shared memory (FP32) and adds
// once per column to the FP64 total.  No FP64 arithmetic per item: the FP64
// pipe of the GB300 SM is a small fraction of its FP32 rate.

constexpr int kShCols = 1024;   // columns combined in shared memory per block

struct ColSum {
    float v[4];
    int p;
    __device__ ColSum() : v{0.f, 0.f, 0.f, 0.f}, p(-1) {}
    __device__ void flush(double* dst) {
        if (p >= 0)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (v[u] != 0.f) atomicAdd(dst + 4 * p + u, (double)v[u]);
        v[0] = v[1] = v[2] = v[3] = 0.f;
    }
    // the thread moves to quad pp (a change only when the grid stride is not
    // a multiple of the quads per node)
    __device__ void at(int pp, double* dst) {
        if (pp != p) {
            flush(dst);
            p = pp;
        }
    }
};

// All threads of the block call this at the same point.
__device__ void colsum_finish(ColSum& cs, double* dst, double* sh, int nc) {
    if (nc > kShCols) {
        cs.flush(dst);
        return;
    }
    float* shf = reinterpret_cast<float*>(sh);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) shf[c] = 0.f;
    __syncthreads();
    if (cs.p >= 0)
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (cs.v[u] != 0.f) atomicAdd(shf + 4 * cs.p + u, cs.v[u]);
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
        if (shf[c] != 0.f) atomicAdd(dst + c, (double)shf[c]);
    __syncthreads();
    cs = ColSum();
}

struct E0Q {   // what the quad phases need of E0Args<float>
    int nRp, m, nSp, nc, nq, nqd;
    double tol2;
    const double* B;
    double* X;
    float *R, *P, *AP, *B0;
    float* X32;                 // the iterate, FP32 (X written once at the end)
    const double* bb;
    MGDeviceLevel L0;
    const float4* wq;
    const unsigned short* ql;   // the iteration's active quads (null: all)
    int na;                     // how many
};

// Lists, in increasing order, the quads that hold a column whose residual is
// still above the tolerance (rr > tol2 bb, the test the per-column tables
// make); every block builds the same list from the same global values.  One
// quad per thread: nq <= blockDim.x.
__device__ int quad_list(int nq, double tol2, const double* bb, const double* rr,
                         unsigned short* ql, int* s_cnt) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    bool on = false;
    if (t < nq)
#pragma unroll
        for (int u = 0; u < 4; ++u)
            on = on || ldg2(rr + 4 * t + u) > tol2 * ldg2(bb + 4 * t + u);
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) s_cnt[w] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int v = 0; v < nw; ++v) {
        const int cv = s_cnt[v];
        if (v < w) off += cv;
        tot += cv;
    }
    if (on) ql[off + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)t;
    __syncthreads();
    return tot;
}


// Per-block table of the columns' CG scalars, built once per phase so that
// the items read a byte and a float from shared memory instead of doing FP64
// comparisons and divisions per item: act[c] = column c active (and, for the
// direction update, still active), coef[c] = alpha or beta.
enum TableKind { kActOnly, kAlpha, kBeta };

__device__ void col_table(TableKind kind, int nc, double tol2, const double* bb,
                          const double* rr_prev, const double* rz_prev, const double* x3,
                          const double* rr_cur, unsigned char* act, float* coef) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        bool a = ldg2(rr_prev + c) > tol2 * ldg2(bb + c);
        float f = 0.f;
        if (kind == kAlpha && a) {
            const double pap = ldg2(x3 + c);   // p.Ap
            f = pap != 0.0 ? (float)(ldg2(rz_prev + c) / pap) : 0.f;
        } else if (kind == kBeta) {
            a = a && ldg2(rr_cur + c) > tol2 * ldg2(bb + c);
            const double ro = ldg2(rz_prev + c);
            f = a && ro != 0.0 ? (float)(ldg2(x3 + c) / ro) : 0.f;   // x3 = rz of this step
        }
        act[c] = a ? 1 : 0;
        if (kind != kActOnly) coef[c] = f;
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned quad_mask(const unsigned char* act, int col) {
    const uchar4 m = *reinterpret_cast<const uchar4*>(act + col);
    return (unsigned)m.x | ((unsigned)m.y << 1) | ((unsigned)m.z << 2) | ((unsigned)m.w << 3);
}

__device__ __forceinline__ float4 sel4(unsigned m, float4 a, float4 b) {
    return make_float4((m & 1u) ? a.x : b.x, (m & 2u) ? a.y : b.y, (m & 4u) ? a.z : b.z,
                       (m & 8u) ? a.w : b.w);
}

// Loop over the (node i, active quad p) items of the CG, each thread on one
// quad as in QUADS (so its per-column sums stay in registers); e4 = float4
// offset in the even layout, m4 = in the V-cycle layout.
#define CGQ(q)                                                                   \
    ColSum cs;                                                                   \
    const unsigned na__ = q.na > 0 ? (unsigned)q.na : 1u;                        \
    const unsigned rows__ = gridDim.x * blockDim.x / na__;                       \
    const unsigned t__ = blockIdx.x * blockDim.x + threadIdx.x;                  \
    const bool on__ = q.na > 0 && t__ < rows__ * na__;                           \
    const int p = on__ ? quad_at(q.ql, (int)(t__ % na__)) : 0;                   \
    const int r = p / q.nqd, k4 = p - r * q.nqd;                                 \
    const int col = 4 * p;                                                       \
    (void)col;                                                                   \
    _Pragma("unroll 1")                                                          \
    for (int i = (int)(t__ / na__); on__ && i < q.nRp; i += (int)rows__) {       \
        const size_t e4 = ((size_t)r * q.nRp + i) * q.nqd + k4;                  \
        const size_t m4 = (size_t)i * q.nq + p;                                  \
        (void)m4;

__device__ __noinline__ void cgq_init(const E0Q& q, double* bbsum, double* sh) {
    CGQ(q)
        const double2* b2 = reinterpret_cast<const double2*>(q.B) + 2 * e4;
        const double2 b01 = __ldcg(b2), b23 = __ldcg(b2 + 1);
        const float4 bf = make_float4((float)b01.x, (float)b01.y, (float)b23.x, (float)b23.y);
        reinterpret_cast<float4*>(q.X32)[e4] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(q.R)[e4] = bf;
        reinterpret_cast<float4*>(q.B0)[m4] = bf;
        cs.at(p, bbsum);
        cs.v[0] = fmaf(bf.x, bf.x, cs.v[0]);
        cs.v[1] = fmaf(bf.y, bf.y, cs.v[1]);
        cs.v[2] = fmaf(bf.z, bf.z, cs.v[2]);
        cs.v[3] = fmaf(bf.w, bf.w, cs.v[3]);
    }
    colsum_finish(cs, bbsum, sh, q.nc);
}

// P = z, rz = r.z (first direction)
__device__ __noinline__ void cgq_first_dir(const E0Q& q, const float* z, double* rz, double* sh) {
    CGQ(q)
        const float4 zv = ldf4q(z, m4), rv = ldf4q(q.R, e4);
        reinterpret_cast<float4*>(q.P)[e4] = zv;
        cs.at(p, rz);
        cs.v[0] = fmaf(rv.x, zv.x, cs.v[0]);
        cs.v[1] = fmaf(rv.y, zv.y, cs.v[1]);
        cs.v[2] = fmaf(rv.z, zv.z, cs.v[2]);
        cs.v[3] = fmaf(rv.w, zv.w, cs.v[3]);
    }
    colsum_finish(cs, rz, sh, q.nc);
}

// AP = E_0 P and p.Ap for the active columns
// The apply loop of one thread's quad (r, k4) over nodes i0, i0 + step, ...:
// AP = E_0 P and the quad's four sums of p.Ap (masked by am).
__device__ __noinline__ float4 ap_quad(const MGDeviceLevel L0, const float4* __restrict__ wq,
                                       int nqd, int k4, unsigned am, int i0, int step, int n,
                                       const float4* __restrict__ Pr, float4* __restrict__ APr) {
    Quad qd;
    qd.load(wq, nqd, k4);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int i = i0; i < n; i += step) {
        float4 dg;
        const float4 y = e0_apply4(L0, qd, Pr, i, k4, nqd, dg);
        const float4 pv = ld4(Pr + (size_t)i * nqd + k4);
        APr[(size_t)i * nqd + k4] = y;
        if (am & 1u) s.x = fmaf(y.x, pv.x, s.x);
        if (am & 2u) s.y = fmaf(y.y, pv.y, s.y);
        if (am & 4u) s.z = fmaf(y.z, pv.z, s.z);
        if (am & 8u) s.w = fmaf(y.w, pv.w, s.w);
    }
    return s;
}

// AP = E_0 P and p.Ap for the active columns (each thread on one quad, as in
// CGQ)
__device__ __noinline__ void cgq_ap(const E0Q& q, const double* rr_prev, double* pap, double* sh,
                                    unsigned char* s_act, float* s_coef) {
    col_table(kActOnly, q.nc, q.tol2, q.bb, rr_prev, nullptr, nullptr, nullptr, s_act, s_coef);
    ColSum cs;
    const unsigned na = q.na > 0 ? (unsigned)q.na : 1u;
    const unsigned rows = gridDim.x * blockDim.x / na;
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = q.na > 0 && t < rows * na ? quad_at(q.ql, (int)(t % na)) : -1;
    const unsigned am = p >= 0 ? quad_mask(s_act, 4 * p) : 0u;
    if (am) {
        const int r = p / q.nqd, k4 = p - r * q.nqd;
        const size_t off = (size_t)r * q.nRp * q.nqd;
        const float4 v = ap_quad(q.L0, q.wq, q.nqd, k4, am, (int)(t / na), (int)rows, q.nRp,
                                 reinterpret_cast<const float4*>(q.P) + off,
                                 reinterpret_cast<float4*>(q.AP) + off);
        cs.at(p, pap);
        cs.v[0] = v.x;
        cs.v[1] = v.y;
        cs.v[2] = v.z;
        cs.v[3] = v.w;
    }
    colsum_finish(cs, pap, sh, q.nc);
}

// x += alpha p, r -= alpha Ap, V-cycle input = r (0 for finished columns)
__device__ __noinline__ void cgq_update(const E0Q& q, const double* rr_prev, const double* rz_prev,
                                        const double* pap, unsigned char* s_act, float* s_coef) {
    col_table(kAlpha, q.nc, q.tol2, q.bb, rr_prev, rz_prev, pap, nullptr, s_act, s_coef);
    CGQ(q)
        const unsigned am = quad_mask(s_act, col);
        float4* b0 = reinterpret_cast<float4*>(q.B0) + m4;
        if (!am) {
            *b0 = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const float4 a4 = *reinterpret_cast<const float4*>(s_coef + col);
        const float al[4] = {a4.x, a4.y, a4.z, a4.w};
        const float4 pv = ldf4q(q.P, e4), rv = ldf4q(q.R, e4), apv = ldf4q(q.AP, e4);
        const float4 xv = ldf4q(q.X32, e4);
        reinterpret_cast<float4*>(q.X32)[e4] =
            make_float4(fmaf(al[0], pv.x, xv.x), fmaf(al[1], pv.y, xv.y),
                        fmaf(al[2], pv.z, xv.z), fmaf(al[3], pv.w, xv.w));
        const float4 rn = make_float4(rv.x - al[0] * apv.x, rv.y - al[1] * apv.y,
                                      rv.z - al[2] * apv.z, rv.w - al[3] * apv.w);
        reinterpret_cast<float4*>(q.R)[e4] = rn;
        *b0 = sel4(am, rn, make_float4(0.f, 0.f, 0.f, 0.f));
    }
}

// rz = r.z and rr = r.r for the active columns; finished columns keep their
// previous values
__device__ __noinline__ void cgq_rz(const E0Q& q, const float* z, const double* rr_prev,
                                    const double* rz_prev, double* rz, double* rr, double* sh,
                                    unsigned char* s_act, float* s_coef) {
    col_table(kActOnly, q.nc, q.tol2, q.bb, rr_prev, nullptr, nullptr, nullptr, s_act, s_coef);
    ColSum c2;
    {
        CGQ(q)
            const unsigned am = quad_mask(s_act, col);
            if (!am) continue;
            const float4 rv = ldf4q(q.R, e4), zv = ldf4q(z, m4);
            cs.at(p, rz);
            c2.at(p, rr);
            const float r4[4] = {rv.x, rv.y, rv.z, rv.w}, z4[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if ((am >> u) & 1u) {
                    cs.v[u] = fmaf(r4[u], z4[u], cs.v[u]);
                    c2.v[u] = fmaf(r4[u], r4[u], c2.v[u]);
                }
        }
        colsum_finish(cs, rz, sh, q.nc);
    }
    colsum_finish(c2, rr, sh, q.nc);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < q.nc; c += gridDim.x * blockDim.x)
        if (!(ldg2(rr_prev + c) > q.tol2 * ldg2(q.bb + c))) {
            rr[c] = ldg2(rr_prev + c);
            rz[c] = ldg2(rz_prev + c);
        }
}

// X (FP64, the caller's layout) = the FP32 iterate, every column
__device__ __noinline__ void cgq_store_x(const E0Q& q) {
    CGQ(q)
        const float4 xv = ldf4q(q.X32, e4);
        double2* x2 = reinterpret_cast<double2*>(q.X) + 2 * e4;
        x2[0] = make_double2((double)xv.x, (double)xv.y);
        x2[1] = make_double2((double)xv.z, (double)xv.w);
    }
}

// p = z + beta p for the columns still active
__device__ __noinline__ void cgq_pupdate(const E0Q& q, const float* z, const double* rr_prev,
                                         const double* rr, const double* rz_prev,
                                         const double* rz, unsigned char* s_act, float* s_coef) {
    col_table(kBeta, q.nc, q.tol2, q.bb, rr_prev, rz_prev, rz, rr, s_act, s_coef);
    CGQ(q)
        const unsigned um = quad_mask(s_act, col);
        if (!um) continue;
        const float4 b4 = *reinterpret_cast<const float4*>(s_coef + col);
        const float be[4] = {b4.x, b4.y, b4.z, b4.w};
        const float4 zv = ldf4q(z, m4), pv = ldf4q(q.P, e4);
        const float4 np = make_float4(zv.x + be[0] * pv.x, zv.y + be[1] * pv.y,
                                      zv.z + be[2] * pv.z, zv.w + be[3] * pv.w);
        reinterpret_cast<float4*>(q.P)[e4] = sel4(um, np, pv);
    }
}
#undef CGQ

__global__ void __launch_bounds__(256, 2) k_e0_pcg_f(E0Args<float> a) {
    __shared__ double sh[kShCols];
    __shared__ __align__(16) float s_coef[kShCols];
    __shared__ __align__(16) unsigned char s_act[kShCols];
    __shared__ unsigned short s_ql[kShCols / 4];
    __shared__ int s_cnt[32];
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = 0;
    E0Q q;
    q.nRp = a.nRp;
    q.m = a.m;
    q.nSp = a.nSp;
    q.nc = a.ncols;
    q.nq = a.ncols >> 2;
    q.nqd = a.nSp >> 2;
    q.tol2 = a.tol2;
    q.B = a.B;
    q.X = a.X;
    q.X32 = a.X32;
    q.R = a.R;
    q.P = a.P;
    q.AP = a.AP;
    q.L0 = a.mg.lev[0];
    q.B0 = q.L0.B;
    q.bb = a.bb;
    q.wq = a.mg.wq;
    q.ql = nullptr;
    q.na = q.nq;
    long long quads_done = q.nq;   // active quads summed over the V-cycles
    const int nc = a.ncols;
    cgq_init(q, a.bb, sh);
    if (!grid_sync(a.bar)) return;
    float* z = nullptr;
    if (!e0_vcycle(a.mg, a.bar, z)) return;
    cgq_first_dir(q, z, slot(a, 2, 1), sh);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
        slot(a, 2, 2)[c] = ldg2(a.bb + c);
    if (!grid_sync(a.bar)) return;
    int it = 0;
    for (; it < a.maxit; ++it) {
        const int cur = it % 3, prev = (it + 2) % 3, next = (it + 1) % 3;
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < 3 * nc; c += blockDim.x)
                a.acc[(size_t)next * 3 * nc + c] = 0.0;
        // every phase of this iteration, the V-cycle included, visits only
        // the quads with an unconverged column
        q.na = quad_list(q.nq, q.tol2, q.bb, slot(a, prev, 2), s_ql, s_cnt);
        q.ql = s_ql;
        quads_done += q.na;
        cgq_ap(q, slot(a, prev, 2), slot(a, cur, 0), sh, s_act, s_coef);
        if (!grid_sync(a.bar)) return;
        cgq_update(q, slot(a, prev, 2), slot(a, prev, 1), slot(a, cur, 0), s_act, s_coef);
        if (!grid_sync(a.bar)) return;
        if (!e0_vcycle(a.mg, a.bar, z, q.ql, q.na)) return;
        cgq_rz(q, z, slot(a, prev, 2), slot(a, prev, 1), slot(a, cur, 1), slot(a, cur, 2), sh,
               s_act, s_coef);
        if (!grid_sync(a.bar)) return;
        cgq_pupdate(q, z, slot(a, prev, 2), slot(a, cur, 2), slot(a, prev, 1), slot(a, cur, 1),
                    s_act, s_coef);
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
    q.ql = nullptr;
    q.na = q.nq;
    cgq_store_x(q);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status->iterations = it;
        a.status->converged = s_stop;
        a.status->active_quads = quads_done;
    }
}

// ============================================================ E_c V-cycle
// E_c work is spread over lane groups: G lanes (8, 16 or 32, the smallest
// power of two that holds d) per (rhs, node) item, 32 / G items per warp;
// lane a of a group owns row a of the item's d values.  Blocks are stored
// transposed, [dir][n][b][a], so the lanes of a group read consecutive words.
struct EcMG {
    int L, nrhs, d, nu, G;
    int Q;                 // Kronecker terms of the levels (0: explicit blocks)
    bool dense;
    const float* cinv;     // [(n_c d)][(n_c d)]
    const float* Gq;       // angular blocks of the terms [Q][d][d] (Q > 0)
    const MGDeviceLevel* lev;   // [L], in device memory
};

// Loop over the (rhs, node) items of an array of nn nodes.  All lanes of a
// warp make the same number of trips (an item past the end has ok == false),
// so group shuffles inside the body stay convergent.  Needs `mg`, `d`, `gpw`
// and `grp` in scope; defines r, i, ok and base (offset of the item's first
// value).
#define GROUP_LOOP(nn)                                                             \
    {                                                                              \
    const unsigned gl_n__ = (unsigned)(nn);                                        \
    const unsigned gl_total__ = (unsigned)mg.nrhs * gl_n__;                        \
    const unsigned gl_stride__ = (gridDim.x * blockDim.x) >> 5;                    \
    for (unsigned gw__ = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;             \
         gw__ * (unsigned)gpw < gl_total__; gw__ += gl_stride__) {                 \
        const unsigned item__ = gw__ * (unsigned)gpw + (unsigned)grp;              \
        const bool ok = item__ < gl_total__;                                       \
        const int r = ok ? (int)(item__ / gl_n__) : 0;                             \
        const int i = ok ? (int)(item__ % gl_n__) : 0;                             \
        const size_t base = ((size_t)r * gl_n__ + i) * d;

// y_a = sum over the 7 stencil directions of (E_c block) x, row a = gl
__device__ __forceinline__ float ec_apply(const MGDeviceLevel& L, const float* x, int r, int i,
                                          int d, int gl, bool act) {
    float y = 0.f;
    if (!act) return y;
    const float* xr = x + (size_t)r * L.n * d;
#pragma unroll
    for (int dir = 0; dir < 7; ++dir) {
        const float* xv = xr + (size_t)nbr(i, dir, L.m, L.n) * d;
        const float* blk = L.val + ((size_t)dir * L.n + i) * d * d + gl;
        for (int b = 0; b < d; ++b) y += __ldg(blk + (size_t)b * d) * ldg2(xv + b);
    }
    return y;
}

// The same product with the level in Kronecker form, sum_q S_q (x) G_q:
// t_q = sum_dir S_q(i, nbr) x_nbr (lane a holds component a), then
// y_a = sum_q sum_b G_q[a][b] t_q[b] with t_q[b] from lane b of the group.
// The stencils are node-major [n][7][Qp]; sG holds the G_q in shared memory.
// Every lane of the warp must call this (shuffles).
constexpr int kEcMaxQ = 16;
__device__ __forceinline__ float ec_apply_kron(const MGDeviceLevel& L, const float* sG, int Q,
                                               const float* x, int r, int i, int d, int G,
                                               int gl, bool act) {
    const int qp4 = (Q + 3) >> 2;
    const float4* sk = reinterpret_cast<const float4*>(L.sv) + (size_t)i * 7 * qp4;
    const float* xr = x + (size_t)r * L.n * d;
    float t[kEcMaxQ];
#pragma unroll
    for (int q = 0; q < kEcMaxQ; ++q) t[q] = 0.f;
#pragma unroll
    for (int dir = 0; dir < 7; ++dir) {
        const float xv = act ? ldg2(xr + (size_t)nbr(i, dir, L.m, L.n) * d + gl) : 0.f;
#pragma unroll
        for (int q4 = 0; q4 < kEcMaxQ / 4; ++q4) {
            if (q4 >= qp4) break;
            const float4 s4 = __ldg(sk + dir * qp4 + q4);
            t[4 * q4 + 0] = fmaf(s4.x, xv, t[4 * q4 + 0]);
            t[4 * q4 + 1] = fmaf(s4.y, xv, t[4 * q4 + 1]);
            t[4 * q4 + 2] = fmaf(s4.z, xv, t[4 * q4 + 2]);
            t[4 * q4 + 3] = fmaf(s4.w, xv, t[4 * q4 + 3]);
        }
    }
    float y = 0.f;
    const int row = act ? gl : 0;
#pragma unroll
    for (int q = 0; q < kEcMaxQ; ++q) {
        if (q >= Q) break;
        const float* g = sG + ((size_t)q * d + row) * d;
        for (int b = 0; b < d; ++b) y = fmaf(g[b], __shfl_sync(0xffffffffu, t[q], b, G), y);
    }
    return act ? y : 0.f;
}

// (D v)_a for the group's vector v (value b held by group lane b)
__device__ __forceinline__ float ec_dmul(const float* D, int d, int G, float v, int gl, bool act) {
    float y = 0.f;
    for (int b = 0; b < d; ++b) {
        const float vb = __shfl_sync(0xffffffffu, v, b, G);
        if (act) y += __ldg(D + (size_t)b * d + gl) * vb;
    }
    return y;
}

// Per-rhs sums: every lane accumulates its own partial while its rhs stays
// the same (a change, only at a right-hand-side boundary, flushes with an
// atomic); rhs_flush then combines the lanes of the block and adds once.
struct RhsSum {
    double v;
    int r;
    __device__ RhsSum() : v(0.0), r(-1) {}
    __device__ void add(double x, int rr, double* dst) {
        if (rr != r) {
            if (r >= 0 && v != 0.0) atomicAdd(dst + r, v);
            v = 0.0;
            r = rr;
        }
        v += x;
    }
};

// All threads of the block call this at the same point.
__device__ void rhs_flush(RhsSum& s, double* dst, double* sh_v, int* sh_r) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rlo = __reduce_min_sync(0xffffffffu, s.r < 0 ? 0x7fffffff : s.r);
    const int rhi = __reduce_max_sync(0xffffffffu, s.r);
    double v = s.v;
    if (rlo == rhi) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            sh_v[warp] = v;
            sh_r[warp] = rhi;
        }
    } else {
        if (s.r >= 0 && v != 0.0) atomicAdd(dst + s.r, v);
        if (lane == 0) sh_r[warp] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        int cur = -1;
        for (int w = 0; w < nw; ++w) {
            if (sh_r[w] < 0) continue;
            if (sh_r[w] != cur) {
                if (cur >= 0) atomicAdd(dst + cur, acc);
                acc = 0.0;
                cur = sh_r[w];
            }
            acc += sh_v[w];
        }
        if (cur >= 0) atomicAdd(dst + cur, acc);
    }
    __syncthreads();
    s.v = 0.0;
    s.r = -1;
}

__device__ bool ec_vcycle(const EcMG& mg, const float* sG, GridBar* bar, float*& z) {
    const int d = mg.d, G = mg.G, gpw = 32 / G;
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G;
    auto apply = [&](const MGDeviceLevel& Lv, const float* x, int r, int i, bool act) {
        return mg.Q ? ec_apply_kron(Lv, sG, mg.Q, x, r, i, d, G, gl, act)
                    : ec_apply(Lv, x, r, i, d, gl, act);
    };
    int cur[kMaxMGLevels];
    for (int l = 0; l < mg.L; ++l) cur[l] = 0;
    auto buf = [&](int l, int which) { return which ? mg.lev[l].Xt : mg.lev[l].X; };
    auto jacobi = [&](int l) -> bool {
        const MGDeviceLevel Lv = mg.lev[l];
        const float* x = buf(l, cur[l]);
        float* xt = buf(l, cur[l] ^ 1);
        GROUP_LOOP(Lv.n)
            const bool act = ok && gl < d;
            const float y = apply(Lv, x, r, i, act);
            const float res = act ? ldg2(Lv.B + base + gl) - y : 0.f;
            const float dx = ec_dmul(Lv.dinv + (size_t)i * d * d, d, G, res, gl, act);
            if (act) xt[base + gl] = ldg2(x + base + gl) + kOmega * dx;
        }}
        cur[l] ^= 1;
        return grid_sync(bar);
    };
    auto first = [&](int l) -> bool {
        const MGDeviceLevel Lv = mg.lev[l];
        float* x = buf(l, 0);
        GROUP_LOOP(Lv.n)
            const bool act = ok && gl < d;
            const float bv = act ? ldg2(Lv.B + base + gl) : 0.f;
            const float dx = ec_dmul(Lv.dinv + (size_t)i * d * d, d, G, bv, gl, act);
            if (act) x[base + gl] = kOmega * dx;
        }}
        cur[l] = 0;
        return grid_sync(bar);
    };
    for (int l = 0; l + 1 < mg.L; ++l) {
        const MGDeviceLevel Lv = mg.lev[l];
        if (!first(l)) return false;
        for (int k = 1; k < mg.nu; ++k)
            if (!jacobi(l)) return false;
        const float* x = buf(l, cur[l]);
        float* t = buf(l, cur[l] ^ 1);
        GROUP_LOOP(Lv.n)
            const bool act = ok && gl < d;
            const float y = apply(Lv, x, r, i, act);
            if (act) t[base + gl] = ldg2(Lv.B + base + gl) - y;
        }}
        if (!grid_sync(bar)) return false;
        const MGDeviceLevel Cv = mg.lev[l + 1];
        GROUP_LOOP(Cv.n)
            if (ok && gl < d) {
                float acc = 0.f;
                for (int q = 0; q < Cv.rwid; ++q) {
                    float w;
                    const int f = restrict_src(Cv, i, q, w);
                    acc += w * ldg2(t + ((size_t)r * Lv.n + f) * d + gl);
                }
                Cv.B[base + gl] = acc;
            }
        }}
        if (!grid_sync(bar)) return false;
    }
    {
        const int l = mg.L - 1;
        const MGDeviceLevel Lv = mg.lev[l];
        if (mg.dense) {
            float* x = buf(l, 0);
            const int N = Lv.n * d;
            // one warp per output entry (rhs, row q): lanes stride over the row
            const unsigned nw = (unsigned)mg.nrhs * N;
            for (unsigned w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
                 w += (gridDim.x * blockDim.x) >> 5) {
                const int r = (int)(w / (unsigned)N), q = (int)(w % (unsigned)N);
                const float* row = mg.cinv + (size_t)q * N;
                const float* b = Lv.B + (size_t)r * N;
                // 6 independent load pairs in flight per lane and trip
                constexpr int U = 6;
                float a4[4] = {0.f, 0.f, 0.f, 0.f};
                int j = lane;
                for (; j + 32 * (U - 1) < N; j += 32 * U) {
                    float rv[U], bv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        rv[u] = __ldg(row + j + 32 * u);
                        bv[u] = ldg2(b + j + 32 * u);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) a4[u % 4] += rv[u] * bv[u];
                }
                for (; j < N; j += 32) a4[0] += __ldg(row + j) * ldg2(b + j);
                float acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) x[(size_t)r * N + q] = acc;
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
        const MGDeviceLevel Lv = mg.lev[l];
        float* x = buf(l, cur[l]);
        const float* xc = buf(l + 1, cur[l + 1]);
        const int ncn = mg.lev[l + 1].n;
        GROUP_LOOP(Lv.n)
            if (ok && gl < d) {
                int c0, c1;
                float w0, w1;
                prolong_src(i, Lv.m, c0, c1, w0, w1);
                const float v = w0 * ldg2(xc + ((size_t)r * ncn + c0) * d + gl) +
                                w1 * ldg2(xc + ((size_t)r * ncn + c1) * d + gl);
                x[base + gl] = ldg2(x + base + gl) + v;
            }
        }}
        if (!grid_sync(bar)) return false;
        for (int k = 0; k < mg.nu; ++k)
            if (!jacobi(l)) return false;
    }
    z = buf(0, cur[0]);
    return true;
}

// ============================================================== E_c PCG
struct EcArgs {
    int nRp, m, d, nrhs, maxit;
    double tol2;
    // direct route (E_c factor): inverses of the row Schur complements
    // [m+1][Bd][ldf] with Bd = (m+1) d, FP32 (mixed modes) or FP64; null
    // on the multigrid route
    const float* lu32;
    const double* lu64;
    int ldf;
    const double* ec;   // FP64 E_c in ELL form, blocks transposed: [7][nRp][b][a]
    const double* B;
    double* X;
    double* R;
    double* P;
    double* AP;
    // FP32 copy of P when the CG's own products run in FP32 on the level-0
    // form of the multigrid (inexact coarse solves), else null
    float* P32;
    double* acc;        // [3][3][nrhs]
    double* bb;
    GridBar* bar;
    SolveStatus* status;
    EcMG mg;
};

// ----------------------------------------- E_c direct route: the sweeps
// E_c is block tridiagonal over the mesh rows y (row blocks of Bd = (m+1) d
// unknowns, node-major, component fastest): A_yy couples a row's nodes
// (self, +x, -x), A_y,y-1 reaches (x, y-1) and (x-1, y-1), A_y,y+1 = its
// transpose.  With the inverses S_y^{-1} of its row Schur complements,
//   forward   w_y = S_y^{-1} (r_y - A_y,y-1 w_y-1)
//   backward  z_y = w_y - S_y^{-1} (A_y,y+1 z_y+1)
// is z = E_c^{-1} r (the exact factorisation: the CG then converges in one
// or two iterations).  Each row takes two grid-wide phases: the couplings
// (one item per unknown) into the scratch row t, then the dense product,
// one output row per warp with the block's copy of t in shared memory.
constexpr int kEcDirectMaxBd = 2400;   // (m+1) d of the largest mesh the route takes
constexpr int kEcSweepRhs = 2;         // right-hand sides staged per product pass

// four consecutive factor entries as floats, streamed
__device__ __forceinline__ float4 ec_ld4(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ec_ld4(const double* p) {
    const double2 u = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    return make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
}

// z[r][y][i] (=, or -= when subtract) sum_j S[i][j] t[r][y][j] for every row i
// of the row block: one warp per output row, 16-byte loads of the (zero-
// padded, ldf a multiple of 4) factor row, the block's copy of t in shared
// memory (zero past Bd).
template <typename T>
__device__ void ec_product(const T* __restrict__ S, int Bd, int ldf, int nrhs, int nRp, int d,
                           int y, int b, const float* t, float* z, bool subtract, float* sv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t rstride = (size_t)nRp * d;   // one right-hand side's vector
    const int q4 = ldf >> 2;
    for (int r0 = 0; r0 < nrhs; r0 += kEcSweepRhs) {
        const int nr = min(kEcSweepRhs, nrhs - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < nr * ldf; e += blockDim.x) {
            const int r = e / ldf, j = e - r * ldf;
            sv[r * ldf + j] = j < Bd ? ldg2(t + (r0 + r) * rstride + (size_t)y * b * d + j) : 0.f;
        }
        __syncthreads();
        for (int i = blockIdx.x * nw + warp; i < Bd; i += gridDim.x * nw) {
            const T* row = S + (size_t)i * ldf;
            float acc[kEcSweepRhs] = {0.f, 0.f};
#pragma unroll 8
            for (int j4 = lane; j4 < q4; j4 += 32) {
                const float4 s4 = ec_ld4(row + 4 * j4);
#pragma unroll
                for (int r = 0; r < kEcSweepRhs; ++r)
                    if (r < nr) {
                        const float4 v4 = reinterpret_cast<const float4*>(sv + r * ldf)[j4];
                        acc[r] = fmaf(s4.x, v4.x, fmaf(s4.y, v4.y, fmaf(s4.z, v4.z,
                                 fmaf(s4.w, v4.w, acc[r]))));
                    }
            }
#pragma unroll
            for (int r = 0; r < kEcSweepRhs; ++r) {
                float v = acc[r];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && r < nr) {
                    float* zp = z + (r0 + r) * rstride + (size_t)y * b * d + i;
                    *zp = subtract ? ldg2(zp) - v : v;
                }
            }
        }
    }
}

// z = E_c^{-1} rin by the factor's two sweeps (all blocks call it).  The
// coupling phases take one unknown per group of 16 lanes, lane c holding
// the coupling column c (d <= 16), summed by shuffles.
__device__ bool ec_sweep(const EcArgs& a, const float* rin, float* t, float* z, GridBar* bar,
                         float* sv) {
    const int d = a.d, b = a.m + 1, Bd = b * d, n = a.nRp;
    const size_t dd = (size_t)d * d, rstride = (size_t)n * d;
    const unsigned items = (unsigned)a.nrhs * Bd;
    const unsigned gstride = (gridDim.x * blockDim.x) >> 4;
    const int c = threadIdx.x & 15;
    // coupling block of node `node`, stencil direction dir, entry (ra, cb)
    auto cpl = [&](int dir, int node, int ra, int cb) {
        return __ldg(a.ec + ((size_t)dir * n + node) * dd + (size_t)cb * d + ra);
    };
    // every lane of a warp makes the same number of trips (shuffles)
    const unsigned trips = (items + gstride - 1) / gstride;
    for (int y = 0; y < b; ++y) {
        unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
        for (unsigned k = 0; k < trips; ++k, e += gstride) {
            const bool ok = e < items;
            const int r = ok ? (int)(e / Bd) : 0, X = ok ? (int)(e % Bd) : 0;
            const int x = X / d, ra = X - x * d;
            const size_t row = r * rstride + (size_t)y * b * d;
            double v = 0.0;
            if (ok && y > 0 && c < d) {
                const int node = y * b + x;
                const float* wp = z + row - (size_t)b * d;   // w_y-1
                v = -cpl(4, node, ra, c) * (double)ldg2(wp + x * d + c);
                if (x > 0) v -= cpl(6, node, ra, c) * (double)ldg2(wp + (x - 1) * d + c);
            }
            for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (ok && c == 0) t[row + X] = (float)(v + (double)ldg2(rin + row + X));
        }
        if (!grid_sync(bar)) return false;
        if (a.lu32) ec_product(a.lu32 + (size_t)y * Bd * a.ldf, Bd, a.ldf, a.nrhs, n, d, y, b, t, z,
                               false, sv);
        else ec_product(a.lu64 + (size_t)y * Bd * a.ldf, Bd, a.ldf, a.nrhs, n, d, y, b, t, z,
                        false, sv);
        if (!grid_sync(bar)) return false;
    }
    for (int y = b - 2; y >= 0; --y) {
        unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
        for (unsigned k = 0; k < trips; ++k, e += gstride) {
            const bool ok = e < items;
            const int r = ok ? (int)(e / Bd) : 0, X = ok ? (int)(e % Bd) : 0;
            const int x = X / d, ra = X - x * d;
            const size_t row = r * rstride + (size_t)y * b * d;
            double v = 0.0;
            if (ok && c < d) {
                const int node = y * b + x;
                const float* zn = z + row + (size_t)b * d;   // z_y+1
                v = cpl(3, node, ra, c) * (double)ldg2(zn + x * d + c);
                if (x + 1 < b) v += cpl(5, node, ra, c) * (double)ldg2(zn + (x + 1) * d + c);
            }
            for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (ok && c == 0) t[row + X] = (float)v;
        }
        if (!grid_sync(bar)) return false;
        if (a.lu32) ec_product(a.lu32 + (size_t)y * Bd * a.ldf, Bd, a.ldf, a.nrhs, n, d, y, b, t, z,
                               true, sv);
        else ec_product(a.lu64 + (size_t)y * Bd * a.ldf, Bd, a.ldf, a.nrhs, n, d, y, b, t, z,
                        true, sv);
        if (!grid_sync(bar)) return false;
    }
    return true;
}

// kDirect: preconditioned by the factor's sweeps (direct route), else by one
// V-cycle; two instantiations so that each route's registers are its own.
template <bool kDirect>
__global__ void __launch_bounds__(256, 4) k_ec_pcg(EcArgs a) {
    __shared__ int s_stop;
    // the direct route's staged row (a single element on the multigrid route)
    __shared__ __align__(16) float s_sv[kDirect ? kEcSweepRhs * kEcDirectMaxBd : 4];
    __shared__ double sh_v[32];
    __shared__ int sh_r[32];
    __shared__ float sG[kEcMaxQ * 16 * 16];   // angular blocks of the Kronecker terms
    if (threadIdx.x == 0) s_stop = 0;
    for (int t = threadIdx.x; t < a.mg.Q * a.d * a.d; t += blockDim.x) sG[t] = __ldg(a.mg.Gq + t);
    __syncthreads();
    const EcMG& mg = a.mg;
    const int d = a.d, G = mg.G, gpw = 32 / G;
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G;
    float* B0 = mg.lev[0].B;
    float* const P32 = kDirect ? nullptr : a.P32;   // FP32 products: multigrid route only
    auto sl = [&](int s, int q) { return a.acc + ((size_t)s * 3 + q) * a.nrhs; };
    RhsSum sum;
    GROUP_LOOP(a.nRp)
        if (ok && gl < d) {
            const double b = a.B[base + gl];
            a.X[base + gl] = 0.0;
            a.R[base + gl] = b;
            B0[base + gl] = (float)b;
            sum.add(b * b, r, a.bb);
        }
    }}
    rhs_flush(sum, a.bb, sh_v, sh_r);
    if (!grid_sync(a.bar)) return;
    // the preconditioner: the factor's sweeps (direct route) or one V-cycle
    auto precondition = [&](float*& zz) -> bool {
        if constexpr (kDirect) {
            zz = mg.lev[0].X;
            return ec_sweep(a, B0, mg.lev[0].Xt, zz, a.bar, s_sv);
        } else {
            return ec_vcycle(mg, sG, a.bar, zz);
        }
    };
    float* z = nullptr;
    if (!precondition(z)) return;
    GROUP_LOOP(a.nRp)
        if (ok && gl < d) {
            const double zv = ldg2(z + base + gl);
            a.P[base + gl] = zv;
            if (P32) P32[base + gl] = (float)zv;
            sum.add(ldg2(a.R + base + gl) * zv, r, sl(2, 1));
        }
    }}
    rhs_flush(sum, sl(2, 1), sh_v, sh_r);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nrhs; c += gridDim.x * blockDim.x)
        sl(2, 2)[c] = ldg2(a.bb + c);
    if (!grid_sync(a.bar)) return;
    int it = 0;
    for (; it < a.maxit; ++it) {
        const int cur = it % 3, prev = (it + 2) % 3, next = (it + 1) % 3;
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < 3 * a.nrhs; c += blockDim.x)
                a.acc[(size_t)next * 3 * a.nrhs + c] = 0.0;
        GROUP_LOOP(a.nRp)
            const bool act = ok && gl < d && ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
            if (P32) {
                // every lane of the warp takes part (the Kronecker form shuffles)
                const float yf = mg.Q ? ec_apply_kron(mg.lev[0], sG, mg.Q, P32, r, i, d, G, gl, act)
                                      : ec_apply(mg.lev[0], P32, r, i, d, gl, act);
                if (act) {
                    a.AP[base + gl] = (double)yf;
                    sum.add((double)yf * ldg2(a.P + base + gl), r, sl(cur, 0));
                }
            } else if (act) {
                double y = 0.0;
                const double* Pr = a.P + (size_t)r * a.nRp * d;
#pragma unroll
                for (int dir = 0; dir < 7; ++dir) {
                    const double* blk = a.ec + ((size_t)dir * a.nRp + i) * d * d + gl;
                    const double* xv = Pr + (size_t)nbr(i, dir, a.m, a.nRp) * d;
                    for (int b = 0; b < d; ++b) y = fma(__ldg(blk + (size_t)b * d), ldg2(xv + b), y);
                }
                a.AP[base + gl] = y;
                sum.add(y * ldg2(a.P + base + gl), r, sl(cur, 0));
            }
        }}
        rhs_flush(sum, sl(cur, 0), sh_v, sh_r);
        if (!grid_sync(a.bar)) return;
        GROUP_LOOP(a.nRp)
            if (ok && gl < d) {
                const bool act = ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
                if (act) {
                    const double pap = ldg2(sl(cur, 0) + r);
                    const double alpha = pap != 0.0 ? ldg2(sl(prev, 1) + r) / pap : 0.0;
                    a.X[base + gl] += alpha * ldg2(a.P + base + gl);
                    const double rv = ldg2(a.R + base + gl) - alpha * ldg2(a.AP + base + gl);
                    a.R[base + gl] = rv;
                    B0[base + gl] = (float)rv;
                    sum.add(rv * rv, r, sl(cur, 2));
                } else {
                    B0[base + gl] = 0.f;
                }
            }
        }}
        rhs_flush(sum, sl(cur, 2), sh_v, sh_r);
        if (!grid_sync(a.bar)) return;
        if (!precondition(z)) return;
        GROUP_LOOP(a.nRp)
            if (ok && gl < d && ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r))
                sum.add(ldg2(a.R + base + gl) * (double)ldg2(z + base + gl), r, sl(cur, 1));
        }}
        rhs_flush(sum, sl(cur, 1), sh_v, sh_r);
        if (!grid_sync(a.bar)) return;
        GROUP_LOOP(a.nRp)
            if (ok) {
                const bool was = ldg2(sl(prev, 2) + r) > a.tol2 * ldg2(a.bb + r);
                if (!was) {
                    if (i == 0 && gl == 0) {
                        sl(cur, 2)[r] = ldg2(sl(prev, 2) + r);
                        sl(cur, 1)[r] = ldg2(sl(prev, 1) + r);
                    }
                } else if (gl < d && ldg2(sl(cur, 2) + r) > a.tol2 * ldg2(a.bb + r)) {
                    const double rzo = ldg2(sl(prev, 1) + r);
                    const double beta = rzo != 0.0 ? ldg2(sl(cur, 1) + r) / rzo : 0.0;
                    const double pv = (double)ldg2(z + base + gl) + beta * ldg2(a.P + base + gl);
                    a.P[base + gl] = pv;
                    if (P32) P32[base + gl] = (float)pv;
                }
            }
        }}
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
#undef GROUP_LOOP

__global__ void k_copy_err(const GridBar* bar, SolveStatus* st) { st->timed_out = bar->err; }

// Blocks per SM of a persistent kernel: as many as fit (the grid barrier
// requires them all to be resident), at most 4.
// A problem with less work takes fewer blocks (one per `per_block` of its
// `units`): its grid barriers are cheaper, and the persistent kernels of
// small solves on other streams (the server's slots) can run beside it.
int coop_grid(const void* fn, int threads, size_t units, size_t per_block) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    per_sm = std::max(1, std::min(per_sm, 4));
    const size_t full = (size_t)per_sm * device_sm_count();
    const size_t want = (units + per_block - 1) / per_block;
    return (int)std::max<size_t>(1, std::min(full, want));
}

template <typename V>
V view(const MGDevice& m) {
    V g{};
    g.L = m.L;
    g.nu = m.nu;
    g.dense = m.dense;
    g.cinv = m.cinv;
    g.lev = m.dev_lev;
    return g;
}

// Optional phase trace of the persistent kernels (set by set_phase_trace).
unsigned long long* g_trace_buf = nullptr;
int g_trace_cap = 0;
// Barrier wait limit of the next launches (0: the default of persist.cuh).
unsigned long long g_wait_limit_ns = 0;

int init_bar(cudaStream_t s, GridBar* bar) {
    GridBar h{};
    h.trace = g_trace_buf;
    h.cap = g_trace_cap;
    h.limit_ns = g_wait_limit_ns;
    RTE_CUDA_TRY(cudaMemcpyAsync(bar, &h, sizeof(GridBar), cudaMemcpyHostToDevice, s));
    return RTE_OK;
}

template <typename T>
int e0_pcg_impl(cudaStream_t s, const DevSystem& d, const T* coef, const double* B, double* X,
                int nrhs, double tol, int maxit, void* work, size_t work_bytes,
                SolveStatus* status_dev) {
    if (work_bytes < e0_cg_work_bytes(d, nrhs))
        return fail(RTE_ERR_ARG, "E_0 CG workspace too small");
    if (nrhs * d.nSp > d.e0mg.cap_cols)
        return fail(RTE_ERR_ARG, "E_0 multigrid sized for fewer RHS");
    const size_t n = (size_t)nrhs * d.nRp * d.nSp;
    const int ncols = nrhs * d.nSp;
    char* p = static_cast<char*>(work);
    E0Args<T> a;
    a.R = carve<T>(p, n);
    a.P = carve<T>(p, n);
    a.AP = carve<T>(p, n);
    a.X32 = carve<float>(p, n);
    a.acc = carve<double>(p, 9 * (size_t)ncols);
    a.bb = carve<double>(p, ncols);
    a.bar = carve<GridBar>(p, 1);
    RTE_CUDA_TRY(cudaMemsetAsync(a.acc, 0, 9 * (size_t)ncols * 8, s));
    RTE_CUDA_TRY(cudaMemsetAsync(a.bb, 0, (size_t)ncols * 8, s));
    RTE_TRY(init_bar(s, a.bar));
    RTE_CUDA_TRY(cudaMemsetAsync(status_dev, 0, sizeof(SolveStatus), s));
    a.nRp = d.nRp;
    a.m = d.e0mg.lev[0].m;
    a.nSp = d.nSp;
    a.nrhs = nrhs;
    a.ncols = ncols;
    a.kTiles = (d.nSp + 31) / 32;
    a.chunks = (d.nRp + kChunk - 1) / kChunk;
    a.units = nrhs * a.kTiles * a.chunks;
    a.maxit = maxit;
    a.tol2 = tol * tol;
    a.coef = coef;
    a.B = B;
    a.X = X;
    a.status = status_dev;
    a.mg = view<E0MG>(d.e0mg);
    a.mg.ncols = ncols;
    a.mg.nSp = d.nSp;
    a.mg.w8 = reinterpret_cast<const float4*>(d.e0mg.w8);
    a.mg.wq = reinterpret_cast<const float4*>(d.e0mg.wq);
    // FP32: the quad kernel when the columns fit its shared per-column tables
    const void* fn = (sizeof(T) == sizeof(float) && ncols <= kShCols) ? (const void*)k_e0_pcg_f
                                                                       : (const void*)k_e0_pcg<T>;
    // level-0 work: (node, column) items, four per thread and sweep (quads)
    const int grid = coop_grid(fn, 256, (size_t)d.nRp * ncols, 256 * 16);
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel(fn, grid, 256, args, 0, s));
    k_copy_err<<<1, 1, 0, s>>>(a.bar, status_dev);
    count_launches(2);
    return RTE_OK;
}

// Self-test of the bounded grid barrier: every block meets the others at
// `rounds` barriers, except block skip_block (when >= 0), which leaves
// before the first one, so the others' waits must run out.  Blocks that pass
// every barrier count themselves in *passed.
__global__ void k_barrier_selftest(GridBar* bar, int skip_block, int rounds, int* passed) {
    if ((int)blockIdx.x == skip_block) return;
    for (int r = 0; r < rounds; ++r)
        if (!grid_sync(bar)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1);
}

}  // namespace

void set_phase_trace(unsigned long long* buf, int cap) {
    g_trace_buf = buf;
    g_trace_cap = cap;
}

void set_wait_limit_ns(unsigned long long ns) { g_wait_limit_ns = ns; }

size_t e0_cg_work_bytes(const DevSystem& d, int nrhs) {
    const size_t n = (size_t)nrhs * d.nRp * d.nSp;
    const size_t ncols = (size_t)nrhs * d.nSp;
    return 3 * (((n * 8) + 255) / 256 * 256) + (((n * 4) + 255) / 256 * 256) +
           ((9 * ncols * 8 + 255) / 256 * 256) + ((ncols * 8 + 255) / 256 * 256) + 256;
}

int e0_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs, double tol,
          int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    return e0_pcg_impl<double>(s, d, d.e0coef, B, X, nrhs, tol, maxit, work, work_bytes,
                               status_dev);
}

int e0_cg_lo(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
             double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev) {
    return e0_pcg_impl<float>(s, d, nullptr, B, X, nrhs, tol, maxit, work, work_bytes,
                              status_dev);
}

size_t coarse_cg_work_bytes(const DevSystem& d, int nrhs) {
    const size_t n = (size_t)nrhs * d.nRp * d.dP;
    return 3 * (((n * 8) + 255) / 256 * 256) + (((n * 4) + 255) / 256 * 256) +
           ((9 * (size_t)nrhs * 8 + 255) / 256 * 256) + (((size_t)nrhs * 8 + 255) / 256 * 256) +
           256;
}

int coarse_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
              double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev,
              bool f32_products) {
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
    a.P32 = carve<float>(p, n);
    a.acc = carve<double>(p, 9 * (size_t)nrhs);
    a.bb = carve<double>(p, nrhs);
    a.bar = carve<GridBar>(p, 1);
    RTE_CUDA_TRY(cudaMemsetAsync(a.acc, 0, 9 * (size_t)nrhs * 8, s));
    RTE_CUDA_TRY(cudaMemsetAsync(a.bb, 0, (size_t)nrhs * 8, s));
    RTE_TRY(init_bar(s, a.bar));
    RTE_CUDA_TRY(cudaMemsetAsync(status_dev, 0, sizeof(SolveStatus), s));
    a.nRp = d.nRp;
    a.m = d.ecmg.lev[0].m;
    a.d = d.dP;
    a.nrhs = nrhs;
    a.maxit = maxit;
    a.tol2 = tol * tol;
    a.ec = d.ec_ell;
    a.B = B;
    a.X = X;
    a.status = status_dev;
    a.lu32 = d.eclu32;
    a.lu64 = d.eclu64;
    a.ldf = ec_direct_ld(d.m, d.dP);
    a.mg = view<EcMG>(d.ecmg);
    a.mg.nrhs = nrhs;
    a.mg.d = d.dP;
    a.mg.G = d.dP <= 8 ? 8 : (d.dP <= 16 ? 16 : 32);
    a.mg.Q = d.ecmg.Q;
    a.mg.Gq = d.ecmg.G;
    if (a.mg.Q > kEcMaxQ || (a.mg.Q > 0 && d.dP > 16))
        return fail(RTE_ERR_ARG, "Kronecker coarse multigrid: at most 16 terms of d <= 16");
    const bool direct = a.lu32 != nullptr || a.lu64 != nullptr;
    // FP32 products need the multigrid's level 0 (the same E_c, checked at
    // set-up to 1e-10 in its Kronecker form)
    if (!f32_products || direct || d.ecmg.L < 1 || d.ecmg.lev[0].n != d.nRp) a.P32 = nullptr;
    const void* fn = direct ? (const void*)k_ec_pcg<true> : (const void*)k_ec_pcg<false>;
    // level-0 work: (rhs, node) items, one per lane group (16 per block)
    const int grid = coop_grid(fn, 256, (size_t)nrhs * d.nRp, 8 * (32 / a.mg.G));
    void* args[] = {&a};
    RTE_CUDA_TRY(cudaLaunchCooperativeKernel(fn, grid, 256, args, 0, s));
    k_copy_err<<<1, 1, 0, s>>>(a.bar, status_dev);
    count_launches(2);
    return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" int rte_barrier_selftest(int blocks, int skip_block, int rounds, void* stream,
                                    int* timed_out, int* passed_blocks) {
    if (blocks < 1 || rounds < 1 || skip_block >= blocks || !timed_out || !passed_blocks)
        return fail(RTE_ERR_ARG, "bad argument");
    constexpr int kThreads = 128;
    int per_sm = 0;
    RTE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_barrier_selftest, kThreads, 0));
    if ((long long)blocks > (long long)per_sm * device_sm_count())
        return fail(RTE_ERR_ARG, "more blocks than can be resident at once");
    cudaStream_t s = (cudaStream_t)stream;
    GridBar* bar = nullptr;
    int* passed = nullptr;
    if (cudaMallocAsync((void**)&bar, sizeof(GridBar), s) != cudaSuccess)
        return fail(RTE_ERR_NOMEM, "barrier self-test allocation");
    if (cudaMallocAsync((void**)&passed, sizeof(int), s) != cudaSuccess) {
        cudaFreeAsync(bar, s);
        return fail(RTE_ERR_NOMEM, "barrier self-test allocation");
    }
    GridBar hb{};
    int rc = RTE_OK;
    if (init_bar(s, bar) != RTE_OK || cudaMemsetAsync(passed, 0, sizeof(int), s) != cudaSuccess)
        rc = fail(RTE_ERR_CUDA, "barrier self-test set-up");
    if (rc == RTE_OK) {
        void* args[] = {&bar, &skip_block, &rounds, &passed};
        count_launches(1);
        if (cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, blocks, kThreads, args,
                                        0, s) != cudaSuccess ||
            cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(passed_blocks, passed, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
            rc = fail(RTE_ERR_CUDA, "barrier self-test launch");
    }
    cudaFreeAsync(bar, s);
    cudaFreeAsync(passed, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == RTE_OK)
        rc = fail(RTE_ERR_CUDA, "barrier self-test synchronisation");
    if (rc != RTE_OK) return rc;
    *timed_out = hb.err;
    if (hb.err) return fail(RTE_ERR_TIMEOUT, "a bounded grid barrier timed out");
    return RTE_OK;
}
