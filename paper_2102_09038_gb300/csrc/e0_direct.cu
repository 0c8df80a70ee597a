// E_0^{-1} by a direct factorisation of its direction blocks, the route of
// the paper's experiments (Section 6: E_0's blocks solved by a sparse direct
// factorisation), laid out for the GPU.
//
// Block k of E_0 (eq. equivalence_bE_bE0) is the 7-point stencil of the
// "/"-mesh with the direction's weights.  With the nodes in lexicographic
// order (x fastest) it is block tridiagonal over the mesh rows y = 0..m, each
// block of size b = m + 1:
//   A_yy      tridiagonal (self, +x, -x),
//   A_y,y-1   two diagonals (-y: node (x, y-1), -x-y: node (x-1, y-1)),
//   A_y,y+1 = A_y+1,y^T.
// Its block LDU factorisation A = L D U has D = diag(S_y) with the Schur
// complements S_0 = A_00, S_y = A_yy - A_y,y-1 S_y-1^{-1} A_y-1,y, and is
// stored as the explicit inverses S_y^{-1} (dense, symmetric, b x b).  The
// solve is then a forward and a backward sweep over the rows, each a dense
// matrix-vector product with S_y^{-1} plus the two-diagonal couplings:
//   forward   w_y = S_y^{-1} (b_y - A_y,y-1 w_y-1)
//   backward  x_y = w_y - S_y^{-1} (A_y,y+1 x_y+1)
// so the solve streams the factor from HBM twice, in wide coalesced loads,
// with one block per direction (and all right-hand sides of the direction
// in that block, so the factor is read once for up to kRB of them).
//
// Setup factorises in FP64 (one block per direction, S_y in shared memory,
// Gauss-Jordan inversion); the factor is kept in FP64 (FP64 mode) or FP32
// (mixed modes, where E_0^{-1} is a preconditioner under the FP64 outer
// residual).
#include <cuda_runtime.h>

#include <algorithm>

#include "device.h"
#include "rte_internal.h"

namespace rte {

namespace {

constexpr int kThreads = 256;
constexpr int kRB = 4;   // right-hand sides per sweep of the factor
// largest mesh of the route: the FP32 solve stages two factor blocks of
// ld x ld floats (ld <= 160) in shared memory beside its vectors
constexpr int kMaxM = 156;
constexpr int kE = 3;    // elements of a [kRB][ld] array per thread (ld <= 160)

// Limit of one wait for a factor block (SM clock cycles; ~2 s at 2 GHz),
// and the flag a wait that ran out sets.
__device__ long long g_e0_wait_cycles = 4000000000ll;
__device__ int g_e0_error = 0;

__device__ __forceinline__ double cf(const double* coef, int nRp, int nSp, int dir, int node,
                                     int k) {
    return coef[((size_t)dir * nRp + node) * nSp + k];
}

// Factorisation of direction block k = blockIdx.x.  G: FP64 scratch of b x b
// per direction (S_y-1^{-1} while S_y is formed); out32 / out64: the inverses,
// [k][y][ld][ld], zero-padded to ld.
__global__ void __launch_bounds__(kThreads) k_e0_factor(int m, int nSp, int ld,
                                                        const double* __restrict__ coef,
                                                        double* __restrict__ G,
                                                        float* __restrict__ out32,
                                                        double* __restrict__ out64) {
    extern __shared__ double sm[];
    const int b = m + 1, nRp = b * b, k = blockIdx.x;
    double* S = sm;                 // b x b, row-major, leading dimension b
    double* colp = S + b * b;       // column p before elimination
    double* rowp = colp + b;        // row p after scaling
    double* Gk = G + (size_t)k * b * b;
    const int bb = b * b;
    for (int y = 0; y < b; ++y) {
        // S_y = A_yy - A_y,y-1 S_y-1^{-1} A_y-1,y
        for (int e = threadIdx.x; e < bb; e += blockDim.x) {
            const int r = e / b, c = e - r * b;
            const int nr = y * b + r;
            double v = 0.0;
            if (r == c) v = cf(coef, nRp, nSp, 0, nr, k);
            else if (c == r + 1) v = cf(coef, nRp, nSp, 1, nr, k);
            else if (c == r - 1) v = cf(coef, nRp, nSp, 2, nr, k);
            if (y > 0) {
                const int nc = y * b + c;
                const double lr0 = cf(coef, nRp, nSp, 4, nr, k);   // (r, y-1)
                const double lr1 = r > 0 ? cf(coef, nRp, nSp, 6, nr, k) : 0.0;   // (r-1, y-1)
                const double lc0 = cf(coef, nRp, nSp, 4, nc, k);
                const double lc1 = c > 0 ? cf(coef, nRp, nSp, 6, nc, k) : 0.0;
                double s = lr0 * lc0 * Gk[r * b + c];
                if (c > 0) s += lr0 * lc1 * Gk[r * b + c - 1];
                if (r > 0) s += lr1 * lc0 * Gk[(r - 1) * b + c];
                if (r > 0 && c > 0) s += lr1 * lc1 * Gk[(r - 1) * b + c - 1];
                v -= s;
            }
            S[e] = v;
        }
        __syncthreads();
        // in-place Gauss-Jordan inversion (S is SPD: no pivoting)
        for (int p = 0; p < b; ++p) {
            const double d = 1.0 / S[p * b + p];
            for (int r = threadIdx.x; r < b; r += blockDim.x) {
                colp[r] = S[r * b + p];
                rowp[r] = r == p ? d : S[p * b + r] * d;
            }
            __syncthreads();
            // (r, c) of entry e advance by the block's stride without a division
            const int sr = blockDim.x / b, sc = blockDim.x - sr * b;
            int r = threadIdx.x / b, c = threadIdx.x - r * b;
            for (int e = threadIdx.x; e < bb; e += blockDim.x) {
                if (r == p) S[e] = rowp[c];
                else if (c == p) S[e] = -colp[r] * d;
                else S[e] = fma(-colp[r], rowp[c], S[e]);
                r += sr;
                c += sc;
                if (c >= b) {
                    c -= b;
                    ++r;
                }
            }
            __syncthreads();
        }
        // symmetrised inverse to the factor and to the scratch of the next row
        const size_t o = ((size_t)k * b + y) * ld * ld;
        for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
            const int r = e / ld, c = e - r * ld;
            const double v = (r < b && c < b) ? 0.5 * (S[r * b + c] + S[c * b + r]) : 0.0;
            if (out32) out32[o + e] = (float)v;
            if (out64) out64[o + e] = v;
            if (r < b && c < b) Gk[r * b + c] = v;
        }
        __syncthreads();
    }
}

// four consecutive factor entries, streamed (each is read once per sweep)
__device__ __forceinline__ void ld4s(const double* p, double (&o)[4]) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 c = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
}

// out[r][x] = sum_c Sinv[c][x] v[r][c] for the nr right-hand sides of the
// sweep (Sinv symmetric: row c read as column c, four consecutive x per
// load).  Thread t takes the four rows 4 (t % nq4) .. + 3 and the column chunk
// t / nq4 of ng; partial sums meet in red.
template <typename T>
__device__ __forceinline__ void matvec(const T* __restrict__ Sinv, int b, int ld, int nr,
                                       const T* v, T* red, T* out) {
    const int nq4 = ld >> 2;
    const int ng = max(1, min(b, (int)blockDim.x / nq4));
    const int cw = (b + ng - 1) / ng;
    const int q = threadIdx.x % nq4, g = threadIdx.x / nq4;
    if (g < ng) {
        T acc[kRB][4];
#pragma unroll
        for (int r = 0; r < kRB; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = T(0);
        const int c0 = g * cw, c1 = min(b, c0 + cw);
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            T s[4];
            ld4s(Sinv + (size_t)c * ld + 4 * q, s);
#pragma unroll
            for (int r = 0; r < kRB; ++r) {
                if (r < nr) {
                    const T vc = v[r * ld + c];
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[r][u] = fma(s[u], vc, acc[r][u]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kRB; ++r)
            if (r < nr)
#pragma unroll
                for (int u = 0; u < 4; ++u) red[((size_t)g * kRB + r) * ld + 4 * q + u] = acc[r][u];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * b; e += blockDim.x) {
        const int r = e / b, x = e - r * b;
        T s = T(0);
        for (int gg = 0; gg < ng; ++gg) s += red[((size_t)gg * kRB + r) * ld + x];
        out[r * ld + x] = s;
    }
    __syncthreads();
}

// X = E_0^{-1} B for direction k = blockIdx.x, every right-hand side, in
// sweeps of kRB right-hand sides.  X holds w_y after the forward sweep.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_e0_direct(int m, int nSp, int nrhs, int ld,
                                                        const T* __restrict__ fac,
                                                        const double* __restrict__ coef,
                                                        const double* __restrict__ B,
                                                        double* __restrict__ X) {
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int b = m + 1, nRp = b * b, k = blockIdx.x;
    T* v = sm;                    // [kRB][ld] right-hand side of the product
    T* prev = v + kRB * ld;       // [kRB][ld] w_y-1 (forward) or x_y+1 (backward)
    T* res = prev + kRB * ld;     // [kRB][ld] the product
    T* red = res + kRB * ld;      // [ng][kRB][ld] partial sums
    const T* fk = fac + (size_t)k * b * ld * ld;
    for (int r0 = 0; r0 < nrhs; r0 += kRB) {
        const int nr = min(kRB, nrhs - r0);
        // forward: w_y = S_y^{-1} (b_y - A_y,y-1 w_y-1)
        for (int y = 0; y < b; ++y) {
            for (int e = threadIdx.x; e < kRB * ld; e += blockDim.x) {
                const int r = e / ld, x = e - r * ld;
                T val = T(0);
                if (r < nr && x < b) {
                    const int node = y * b + x;
                    val = (T)B[((size_t)(r0 + r) * nRp + node) * nSp + k];
                    if (y > 0) {
                        val -= (T)cf(coef, nRp, nSp, 4, node, k) * prev[r * ld + x];
                        if (x > 0) val -= (T)cf(coef, nRp, nSp, 6, node, k) * prev[r * ld + x - 1];
                    }
                }
                v[e] = val;
            }
            __syncthreads();
            matvec<T>(fk + (size_t)y * ld * ld, b, ld, nr, v, red, res);
            for (int e = threadIdx.x; e < kRB * ld; e += blockDim.x) {
                const int r = e / ld, x = e - r * ld;
                prev[e] = res[e];
                if (r < nr && x < b)
                    X[((size_t)(r0 + r) * nRp + y * b + x) * nSp + k] = (double)res[e];
            }
            __syncthreads();
        }
        // backward: x_m = w_m (held in prev); x_y = w_y - S_y^{-1} (A_y,y+1 x_y+1)
        for (int y = b - 2; y >= 0; --y) {
            for (int e = threadIdx.x; e < kRB * ld; e += blockDim.x) {
                const int r = e / ld, x = e - r * ld;
                T val = T(0);
                if (r < nr && x < b) {
                    const int node = y * b + x;
                    val = (T)cf(coef, nRp, nSp, 3, node, k) * prev[r * ld + x];
                    if (x + 1 < b) val += (T)cf(coef, nRp, nSp, 5, node, k) * prev[r * ld + x + 1];
                }
                v[e] = val;
            }
            __syncthreads();
            matvec<T>(fk + (size_t)y * ld * ld, b, ld, nr, v, red, res);
            for (int e = threadIdx.x; e < kRB * ld; e += blockDim.x) {
                const int r = e / ld, x = e - r * ld;
                T xv = T(0);
                if (r < nr && x < b) {
                    double* p = X + ((size_t)(r0 + r) * nRp + y * b + x) * nSp + k;
                    xv = (T)(*p) - res[e];
                    *p = (double)xv;
                }
                prev[e] = xv;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------
// FP32 solve with the factor staged in shared memory by TMA bulk copies (one
// copy per half block, each into its own slot, so copies overlap the
// products).  The blocks are used in the order y = 0..m (forward) then
// m-1..0 (backward): step t takes block t < b ? t : 2b - 2 - t.  The
// right-hand side, the coupling coefficients and (backward) the forward
// result of the next step are loaded into registers one step ahead.

__device__ __forceinline__ uint32_t sh_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait for the phase of parity `par` of the mbarrier at `bar`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t par) {
    const long long t0 = clock64(), lim = g_e0_wait_cycles;
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(par)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > lim) {
            atomicExch(&g_e0_error, 1);
            return false;
        }
    }
}

// Thread 0: one bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) from global src into shared dst, completing on bar.
__device__ __forceinline__ void tma_block(void* dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(sh_addr(dst)), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// The block's product in two halves of its rows c (the columns of the
// product, S being symmetric): half h covers c in [h hb, min(b, (h + 1) hb)),
// hb = ceil(b / 2), contiguous in memory.  Each half goes through its own
// shared-memory slot, so the copy of one half of the next block runs while
// the other half is used, and a block needs about half the shared memory of
// a whole one: two blocks of threads fit on an SM.
__device__ __forceinline__ void matvec_half(const float* __restrict__ S, int c_lo, int c_hi,
                                            int ld, int nr, int q, int g, int cw,
                                            const float* v, float (&acc)[kRB][4]) {
    const int c0 = max(c_lo, g * cw), c1 = min(c_hi, (g + 1) * cw);
#pragma unroll 4
    for (int c = c0; c < c1; ++c) {
        const float4 sv = *reinterpret_cast<const float4*>(S + (size_t)(c - c_lo) * ld + 4 * q);
#pragma unroll
        for (int r = 0; r < kRB; ++r)
            if (r < nr) {
                const float vc = v[r * ld + c];
                acc[r][0] = fmaf(sv.x, vc, acc[r][0]);
                acc[r][1] = fmaf(sv.y, vc, acc[r][1]);
                acc[r][2] = fmaf(sv.z, vc, acc[r][2]);
                acc[r][3] = fmaf(sv.w, vc, acc[r][3]);
            }
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_e0_direct_tma(int m, int nSp, int nrhs, int ld,
                                                               const float* __restrict__ fac,
                                                               const double* __restrict__ coef,
                                                               const double* __restrict__ B,
                                                               double* __restrict__ X) {
    extern __shared__ __align__(128) unsigned char smraw[];
    const int b = m + 1, nRp = b * b, k = blockIdx.x;
    const int hb = (b + 1) / 2;                     // rows of the first half
    const size_t blk = (size_t)ld * ld, slot_elems = (size_t)hb * ld;
    float* slot = reinterpret_cast<float*>(smraw);  // [2][hb][ld]
    float* v = slot + 2 * slot_elems;               // [kRB][ld]
    float* prev = v + kRB * ld;                     // [kRB][ld]
    float* res = prev + kRB * ld;                   // [kRB][ld]
    float* red = res + kRB * ld;                    // [ng][kRB][ld]
    __shared__ __align__(8) unsigned long long bars[2];
    const uint32_t bar[2] = {sh_addr(&bars[0]), sh_addr(&bars[1])};
    const float* fk = fac + (size_t)k * b * blk;
    const int steps = 2 * b - 1;
    auto block_of = [&](int t) { return t < b ? t : 2 * b - 2 - t; };
    // half h of the block of step t: source and byte count
    auto half_src = [&](int t, int h) { return fk + (size_t)block_of(t) * blk + (size_t)h * slot_elems; };
    auto half_bytes = [&](int h) {
        return (uint32_t)((size_t)(h == 0 ? hb : b - hb) * ld * sizeof(float));
    };
    const int nq4 = ld >> 2;
    const int ng = max(1, min(b, (int)blockDim.x / nq4));
    const int cw = (b + ng - 1) / ng;
    const int q = threadIdx.x % nq4, g = threadIdx.x / nq4;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar[0]) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar[1]) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned uses = 0;   // completed phases of each slot's barrier (equal for both)
    for (int r0 = 0; r0 < nrhs; r0 += kRB) {
        const int nr = min(kRB, nrhs - r0);
        if (threadIdx.x == 0) {
            // the previous sweep's reads of both slots are done (its last
            // barrier); order them before the copies' writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_block(slot, half_src(0, 0), half_bytes(0), bar[0]);
            if (b > hb) tma_block(slot + slot_elems, half_src(0, 1), half_bytes(1), bar[1]);
        }
        // registers for step t: B (forward) or the forward result w (backward),
        // and the two coupling coefficients of the row
        double pb[kE], pc0[kE], pc1[kE];
        auto fetch = [&](int t) {
            const bool fw = t < b;
            const int y = block_of(t);
#pragma unroll
            for (int j = 0; j < kE; ++j) {
                const int e = threadIdx.x + j * kThreads;
                const int r = e / ld, x = e - r * ld;
                pb[j] = pc0[j] = pc1[j] = 0.0;
                if (e < kRB * ld && r < nr && x < b) {
                    const int node = y * b + x;
                    if (fw) {
                        pb[j] = B[((size_t)(r0 + r) * nRp + node) * nSp + k];
                        if (y > 0) {
                            pc0[j] = cf(coef, nRp, nSp, 4, node, k);
                            if (x > 0) pc1[j] = cf(coef, nRp, nSp, 6, node, k);
                        }
                    } else {
                        pb[j] = X[((size_t)(r0 + r) * nRp + node) * nSp + k];
                        pc0[j] = cf(coef, nRp, nSp, 3, node, k);
                        if (x + 1 < b) pc1[j] = cf(coef, nRp, nSp, 5, node, k);
                    }
                }
            }
        };
        fetch(0);
        for (int t = 0; t < steps; ++t) {
            const bool fw = t < b;
            const int y = block_of(t);
            // the product's right-hand side from the registers and prev
#pragma unroll
            for (int j = 0; j < kE; ++j) {
                const int e = threadIdx.x + j * kThreads;
                if (e >= kRB * ld) continue;
                const int r = e / ld, x = e - r * ld;
                float val = 0.f;
                if (r < nr && x < b) {
                    if (fw) {
                        val = (float)pb[j];
                        if (y > 0) {
                            val -= (float)pc0[j] * prev[r * ld + x];
                            if (x > 0) val -= (float)pc1[j] * prev[r * ld + x - 1];
                        }
                    } else {
                        val = (float)pc0[j] * prev[r * ld + x];
                        if (x + 1 < b) val += (float)pc1[j] * prev[r * ld + x + 1];
                    }
                }
                v[e] = val;
            }
            // the backward epilogue needs this step's w: keep it before the
            // registers move on to the next step
            float wv[kE];
#pragma unroll
            for (int j = 0; j < kE; ++j) wv[j] = (float)pb[j];
            if (t + 1 < steps) fetch(t + 1);
            __syncthreads();
            float acc[kRB][4];
#pragma unroll
            for (int r = 0; r < kRB; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
            for (int h = 0; h < 2; ++h) {
                const int c_lo = h * hb, c_hi = h == 0 ? hb : b;
                if (c_hi <= c_lo) continue;
                const bool ok = mbar_wait(bar[h], uses & 1u);
                if (__syncthreads_or(!ok)) {
                    // a copy did not arrive in time: let the other slot's copy
                    // finish (bounded) and leave; the host reads g_e0_error
                    if (threadIdx.x == 0 && h == 0 && b > hb) mbar_wait(bar[1], uses & 1u);
                    return;
                }
                if (g < ng) matvec_half(slot + h * slot_elems, c_lo, c_hi, ld, nr, q, g, cw, v, acc);
                __syncthreads();
                if (threadIdx.x == 0 && t + 1 < steps) {
                    // every thread's reads of this slot are done (barrier above)
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_block(slot + h * slot_elems, half_src(t + 1, h), half_bytes(h), bar[h]);
                }
            }
            ++uses;
            if (g < ng)
#pragma unroll
                for (int r = 0; r < kRB; ++r)
                    if (r < nr)
                        *reinterpret_cast<float4*>(red + ((size_t)g * kRB + r) * ld + 4 * q) =
                            make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            __syncthreads();
            for (int e = threadIdx.x; e < nr * ld; e += blockDim.x) {
                float sum = 0.f;
                const int r = e / ld, x = e - r * ld;
                for (int gg = 0; gg < ng; ++gg) sum += red[((size_t)gg * kRB + r) * ld + x];
                res[r * ld + x] = sum;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kE; ++j) {
                const int e = threadIdx.x + j * kThreads;
                if (e >= kRB * ld) continue;
                const int r = e / ld, x = e - r * ld;
                float out = 0.f;
                if (r < nr && x < b) {
                    out = fw ? res[e] : wv[j] - res[e];
                    X[((size_t)(r0 + r) * nRp + y * b + x) * nSp + k] = (double)out;
                }
                prev[e] = out;
            }
            __syncthreads();
        }
    }
}

int e0_ld(int m) { return (m + 1 + 3) & ~3; }

template <typename T>
size_t solve_smem(int m) {
    const int ld = e0_ld(m), nq4 = ld / 4;
    const int ng = std::max(1, std::min(m + 1, kThreads / nq4));
    return (size_t)(3 + ng) * kRB * ld * sizeof(T);
}

// the FP32 solve: two staged half blocks and the vectors
size_t tma_smem(int m) {
    const size_t ld = e0_ld(m), hb = (m + 2) / 2;
    return 2 * hb * ld * sizeof(float) + solve_smem<float>(m);
}

}  // namespace

// m <= 156: the FP32 solve's two staged blocks and vectors fit in 227 KB of
// shared memory (and the FP64 set-up's Schur complement in 200 KB).
bool e0_direct_fits(int m) { return m >= 1 && m <= kMaxM; }

size_t e0_direct_bytes(int m, int nSp, bool fp64) {
    const size_t ld = e0_ld(m);
    return (size_t)nSp * (m + 1) * ld * ld * (fp64 ? 8 : 4);
}

size_t e0_direct_scratch_bytes(int m, int nSp) {
    return (size_t)nSp * (m + 1) * (m + 1) * sizeof(double);
}

// Largest dynamic shared memory of a kernel over every mesh the route takes:
// the attribute is per device and per kernel, so every call (from any host
// thread, for any mesh) sets the same value and no call can shrink it under
// another's launch.
size_t factor_smem(int m) { return (size_t)((m + 1) * (m + 1) + 2 * (m + 1)) * sizeof(double); }
template <typename T>
size_t max_solve_smem() {
    size_t mx = 0;
    for (int m = 1; m <= kMaxM; ++m) mx = std::max(mx, solve_smem<T>(m));
    return mx;
}
size_t max_tma_smem() {
    size_t mx = 0;
    for (int m = 1; m <= kMaxM; ++m) mx = std::max(mx, tma_smem(m));
    return mx;
}

int e0_direct_factor(cudaStream_t s, const DevSystem& d, double* scratch, float* out32,
                     double* out64) {
    const int m = d.m;
    if (!e0_direct_fits(m)) return fail(RTE_ERR_ARG, "mesh too large for the direct E_0 route");
    const size_t sm = factor_smem(m);
    RTE_CUDA_TRY(cudaFuncSetAttribute(k_e0_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)factor_smem(kMaxM)));
    count_launches(1);
    k_e0_factor<<<d.nSp, kThreads, sm, s>>>(m, d.nSp, e0_ld(m), d.e0coef, scratch, out32, out64);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int e0_direct_solve(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
                    bool fp64) {
    const int m = d.m, ld = e0_ld(m);
    if (fp64) {
        if (!d.e0lu64) return fail(RTE_ERR_ARG, "no FP64 direct E_0 factor");
        const size_t sm = solve_smem<double>(m);
        RTE_CUDA_TRY(cudaFuncSetAttribute(k_e0_direct<double>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)max_solve_smem<double>()));
        k_e0_direct<double><<<d.nSp, kThreads, sm, s>>>(m, d.nSp, nrhs, ld, d.e0lu64, d.e0coef,
                                                        B, X);
    } else {
        if (!d.e0lu32) return fail(RTE_ERR_ARG, "no FP32 direct E_0 factor");
        const size_t sm = tma_smem(m);
        RTE_CUDA_TRY(cudaFuncSetAttribute(k_e0_direct_tma,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)max_tma_smem()));
        k_e0_direct_tma<<<d.nSp, kThreads, sm, s>>>(m, d.nSp, nrhs, ld, d.e0lu32, d.e0coef, B, X);
    }
    count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int e0_direct_error(cudaStream_t s) {
    int e = 0;
    RTE_CUDA_TRY(cudaMemcpyFromSymbolAsync(&e, g_e0_error, sizeof(int), 0, cudaMemcpyDeviceToHost,
                                           s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) {
        const int zero = 0;
        cudaMemcpyToSymbolAsync(g_e0_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
        return fail(RTE_ERR_TIMEOUT, "a wait for a staged E_0 factor block timed out");
    }
    return RTE_OK;
}

int e0_set_wait_cycles(long long cycles) {
    RTE_CUDA_TRY(cudaMemcpyToSymbol(g_e0_wait_cycles, &cycles, sizeof(cycles)));
    return RTE_OK;
}

}  // namespace rte
