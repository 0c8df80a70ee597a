// Tensor-core GEMM for sm_103a (tcgen05 + TMA) for the dense angular
// contractions of the hot path: the scattering apply U S^+ (eq. bKebKo) and
// the two eigenbasis contractions of (M^- - K^-)^{-1} (Lemma
// apply_high_order_pre taken over the full eigenbasis).
//
//   C[M x N] = epi(A[M x K] * B^T)   with A row-major (K contiguous) and the
//   second operand given K-major as Bt[N x K] (K contiguous)
//
// Operands are BF16 (tcgen05.mma kind::f16) or FP32 read as TF32
// (kind::tf32); accumulation is FP32 in tensor memory.  One CTA computes one
// 128 x BN tile: warp 0 lane 0 issues TMA loads into a 4-stage shared-memory
// ring (128-byte swizzle), warp 1 lane 0 issues the MMAs, and all four warps
// then drain the accumulator with tcgen05.ld and apply the epilogue.  Every
// wait on an mbarrier is bounded: on timeout the kernel records an error flag
// and leaves instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "device.h"
#include "rte_internal.h"
#include "tc_gemm.h"
#include "tcgen05.cuh"

namespace rte {

namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kStages = 4;

template <int BN, bool TF32, typename TOut>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          int M, int N, int K, TOut* __restrict__ C, int ldc, int epi,
          const float* __restrict__ at, const float* __restrict__ as,
          const float* __restrict__ lam, int rows, float beta) {
    constexpr uint32_t kABytes = kBM * kRowBytes;
    constexpr uint32_t kBBytes = BN * kRowBytes;
    constexpr uint32_t kTmemCols = BN;   // FP32 accumulator: one column per N
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment of the operand ring (swizzle atoms)
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int kblocks = (K + (TF32 ? 32 : 64) - 1) / (TF32 ? 32 : 64);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages),
                   done = smem_u32(bars + 2 * kStages);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
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
        // ------------------------------------------------ TMA producer
        for (int kb = 0; kb < kblocks && ok; ++kb) {
            const int s = kb % kStages;
            const uint32_t ph = (kb / kStages) & 1;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1)) { ok = false; break; }
            mbar_expect_tx(full0 + 8 * s, kABytes + kBBytes);
            const int kx = kb * (TF32 ? 32 : 64);
            tma_load_2d(smem_u32(sA + s * kABytes), &mapA, full0 + 8 * s, kx, m0);
            tma_load_2d(smem_u32(sB + s * kBBytes), &mapB, full0 + 8 * s, kx, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------- MMA issuer
        uint32_t idesc = (1u << 4)                                   // D: FP32
                         | ((TF32 ? 2u : 1u) << 7)                   // A: TF32 / BF16
                         | ((TF32 ? 2u : 1u) << 10)                  // B: TF32 / BF16
                         | ((uint32_t)(BN >> 3) << 17)               // N
                         | ((uint32_t)(kBM >> 4) << 24);             // M
        for (int kb = 0; kb < kblocks && ok; ++kb) {
            const int s = kb % kStages;
            const uint32_t ph = (kb / kStages) & 1;
            if (!mbar_wait(full0 + 8 * s, ph)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // 4 MMAs of 32 bytes of K each
                mma_issue(TF32, tmem, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk), idesc,
                          (kb > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(empty0 + 8 * s);   // frees the stage once these MMAs have read it
        }
        mma_commit(done);
    }
    __syncwarp();
    // ---------------------------------------------------------- epilogue
    ok = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    float fat = 0.f, fas = 0.f;
    if (epi != 0 && row < M) {
        const int rr = row % rows;
        fat = at[rr];
        fas = as[rr];
    }
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        // every lane of the warp takes part in the load, whatever its row
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (!ok || row >= M) continue;
        TOut* dst = C + (size_t)row * ldc + n0 + c0;
        const bool full = n0 + c0 + 16 <= N && beta == 0.f &&
                          ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
        if (full) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (epi == 1) v[i] = v[i] / (fat - lam[n0 + c0 + i] * fas);
            if constexpr (sizeof(TOut) == 4) {
                float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            } else {
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                    w[i] = *reinterpret_cast<uint32_t*>(&h);
                }
                uint4* d4 = reinterpret_cast<uint4*>(dst);
                d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
                d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
            continue;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int col = n0 + c0 + i;
            if (col >= N) break;
            float x = v[i];
            if (epi == 1) x = x / (fat - lam[col] * fas);
            if (beta != 0.f) x += beta * static_cast<float>(dst[i]);
            dst[i] = static_cast<TOut>(x);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

template <int BN>
constexpr size_t smem_bytes() {
    return 1024 + (size_t)kStages * (kBM + BN) * kRowBytes + (2 * kStages + 1) * 8 + 16;
}

template <int BN, bool TF32, typename TOut>
int launch(cudaStream_t s, const TcGemmArgs& g) {
    CUtensorMap ma, mb;
    RTE_TRY(make_map(&ma, g.A, TF32, g.M, g.K, kBM));
    RTE_TRY(make_map(&mb, g.Bt, TF32, g.N, g.K, BN));
    auto kern = k_tc_gemm<BN, TF32, TOut>;
    const size_t sm = smem_bytes<BN>();
    // set on every call: the attribute is per device, and cheap to set
    RTE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((g.N + BN - 1) / BN, (g.M + kBM - 1) / kBM);
    count_launches(1);
    kern<<<grid, 128, sm, s>>>(ma, mb, g.M, g.N, g.K, static_cast<TOut*>(g.C), g.ldc, g.epi,
                               g.at, g.as, g.lam, g.rows, g.beta);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

}  // namespace

int tc_gemm(cudaStream_t s, const TcGemmArgs& g) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return RTE_OK;
    if (g.bn != 0 && g.bn != 128 && g.bn != 256) return fail(RTE_ERR_ARG, "tile width 128 or 256");
    const bool wide = g.bn ? g.bn == 256 : g.N > 128;
    if (g.tf32) {
        if (g.out_bf16) return fail(RTE_ERR_ARG, "TF32 GEMM writes FP32");
        return wide ? launch<256, true, float>(s, g) : launch<128, true, float>(s, g);
    }
    if (g.out_bf16)
        return wide ? launch<256, false, __nv_bfloat16>(s, g)
                    : launch<128, false, __nv_bfloat16>(s, g);
    return wide ? launch<256, false, float>(s, g) : launch<128, false, float>(s, g);
}

int tc_set_wait_cycles(long long cycles) {
    RTE_CUDA_TRY(cudaMemcpyToSymbol(g_tc_wait_cycles, &cycles, sizeof(cycles)));
    return RTE_OK;
}

int tc_gemm_error(cudaStream_t s) {
    int e = 0;
    RTE_CUDA_TRY(cudaMemcpyFromSymbolAsync(&e, g_tc_error, sizeof(int), 0,
                                           cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    if (e) {
        const int zero = 0;
        cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
        return fail(RTE_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
    }
    return RTE_OK;
}

}  // namespace rte

// ======================================================================
// FP64-accurate GEMM from exact BF16 tensor-core products (error-free
// splitting of the operands, after Ozaki, Ogita, Oishi and Rump).
//
// Every row of A (and of the K-major second operand Bt) is scaled by a power
// of two 2^e so that its entries lie in (-1, 1), then cut into S balanced
// base-128 digits d_s (|d_0| <= 128, |d_s| <= 64 for s > 0): A = 2^e sum_s
// d_s 2^{-7(s+1)} up to a remainder below 2^{-7S-1}.  Slice s is stored
// scaled, d_s 2^{-7s} (exact in BF16), so that a slice-pair product carries
// its weight 2^{-7(s+t)} itself and
//   A Bt^T = 2^(ea + eb - 14) sum_w P_w,   P_w = sum_{s + t = w} A_s B_t
// over w <= S - 1 (pairs with s + t >= S lie below the truncation level).
// The tensor cores add each 16-term product group to an FP32 accumulator
// with a truncating rounding, whose bias grows with the number of additions:
// so each weight w <= 4 has its own accumulator, in which every partial sum
// over at most 512 terms of K is an exact multiple of 2^{-7w} below 2^{24-7w}
// (each term of P_w at most 28672 2^{-7w}); these are folded into FP64
// registers once per 512 of K.  The weights w >= 5 (S >= 6) share one FP32
// accumulator over the whole K: at most 2^{-35} of the result, so its
// rounding stays near 2^{-58}.
// ======================================================================
namespace rte {

namespace {

using namespace tc;

constexpr int kOzBM = 128, kOzBN = 64, kOzKChunk = 8;     // 8 x 64 = 512 of K per fold
constexpr int kOzMaxS = 9;
constexpr int kOzAcc = 6;                                   // P_0 .. P_4 exact, P_5+ FP32
constexpr uint32_t kOzATile = kOzBM * kRowBytes;            // 16 KB: one A slice tile
constexpr uint32_t kOzBTile = kOzBN * kRowBytes;            // 8 KB: one B slice tile
constexpr uint32_t kOzTmemCols = 512;                       // 6 x 64 columns used

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 18 warps: warp 0 issues TMA loads, warp 1 issues MMAs, warps 2..17 drain
// the accumulators (warp w reads TMEM lanes 32 (w % 4) .. + 31 and the
// quarter (w - 2) / 4 of the 64 columns of each accumulator).
constexpr int kOzThreads = 576;
constexpr int kOzEpiWarps = 16;

// Per 64-wide K block the producer loads the S slices of the B tile into one
// of nB resident sets, then streams the S slices of the A tile through a
// ring of nA slots; the MMA issuer multiplies A slice s with B slices
// t = 0 .. S-1-s into P_{min(s+t, 5)}.  Each tile of A and B is read once per
// K block (the pair products reuse them from shared memory).
__global__ void __launch_bounds__(kOzThreads, 1)
k_ozaki(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
        int M, int N, int K, int S, int nA, int nB, const int* __restrict__ ea,
        const int* __restrict__ eb, double* __restrict__ C, int ldc, int epi,
        const double* __restrict__ at, const double* __restrict__ as,
        const double* __restrict__ lam, int rows) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                                  // nA tiles of 16 KB
    uint8_t* sB = smem + (size_t)nA * kOzATile;          // nB sets of S tiles of 8 KB
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + (size_t)nB * S * kOzBTile);
    // fullA[4], emptyA[4], fullB[2], emptyB[2], accf, acce
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 14);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kOzBM, n0 = blockIdx.x * kOzBN;
    const int kblocks = (K + 63) / 64;
    const int nchunks = (kblocks + kOzKChunk - 1) / kOzKChunk;
    const uint32_t fullA0 = smem_u32(bars), emptyA0 = smem_u32(bars + 4),
                   fullB0 = smem_u32(bars + 8), emptyB0 = smem_u32(bars + 10),
                   accf = smem_u32(bars + 12), acce = smem_u32(bars + 13);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) {
            mbar_init(fullA0 + 8 * i, 1);
            mbar_init(emptyA0 + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(fullB0 + 8 * i, 1);
            mbar_init(emptyB0 + 8 * i, 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, kOzEpiWarps);   // one arrival per epilogue warp
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kOzTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // --------------------------------------------- TMA producer
        int ga = 0;
        for (int kb = 0; kb < kblocks && ok; ++kb) {
            const int sb = kb % nB;
            const uint32_t phb = (kb / nB) & 1;
            if (!mbar_wait(emptyB0 + 8 * sb, phb ^ 1)) { ok = false; break; }
            mbar_expect_tx(fullB0 + 8 * sb, (uint32_t)S * kOzBTile);
            for (int t = 0; t < S; ++t)
                tma_load_2d(smem_u32(sB + ((size_t)sb * S + t) * kOzBTile), &mapB,
                            fullB0 + 8 * sb, kb * 64, t * N + n0);
            for (int s = 0; s < S && ok; ++s, ++ga) {
                const int sa = ga % nA;
                const uint32_t pha = (ga / nA) & 1;
                if (!mbar_wait(emptyA0 + 8 * sa, pha ^ 1)) { ok = false; break; }
                mbar_expect_tx(fullA0 + 8 * sa, kOzATile);
                tma_load_2d(smem_u32(sA + (size_t)sa * kOzATile), &mapA, fullA0 + 8 * sa, kb * 64,
                            s * M + m0);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------- MMA issuer
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(kOzBN >> 3) << 17) | ((uint32_t)(kOzBM >> 4) << 24);
        int ga = 0;
        unsigned started = 0;   // bit a: accumulator a holds a partial sum
        for (int kb = 0; kb < kblocks && ok; ++kb) {
            const int chunk = kb / kOzKChunk;
            if (kb % kOzKChunk == 0) {
                if (chunk > 0) {
                    // the exact accumulators of the previous chunk drained
                    if (!mbar_wait(acce, (chunk - 1) & 1)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                started &= 1u << (kOzAcc - 1);
            }
            const int sb = kb % nB;
            const uint32_t phb = (kb / nB) & 1;
            if (!mbar_wait(fullB0 + 8 * sb, phb)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t b0 = smem_u32(sB + (size_t)sb * S * kOzBTile);
            for (int s = 0; s < S && ok; ++s, ++ga) {
                const int sa = ga % nA;
                const uint32_t pha = (ga / nA) & 1;
                if (!mbar_wait(fullA0 + 8 * sa, pha)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(sA + (size_t)sa * kOzATile);
                for (int t = 0; s + t <= S - 1; ++t) {
                    const int acc = s + t < kOzAcc - 1 ? s + t : kOzAcc - 1;
                    const uint32_t dtm = tmem + (uint32_t)(acc * kOzBN);
                    const uint32_t bt = b0 + (uint32_t)t * kOzBTile;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_issue(false, dtm, sw128_desc(a0 + 32 * kk), sw128_desc(bt + 32 * kk),
                                  idesc, (((started >> acc) & 1u) || kk > 0) ? 1u : 0u);
                    started |= 1u << acc;
                }
                mma_commit(emptyA0 + 8 * sa);   // frees the A slot once its MMAs have read it
            }
            mma_commit(emptyB0 + 8 * sb);
            if (kb % kOzKChunk == kOzKChunk - 1 || kb == kblocks - 1) mma_commit(accf);
        }
    }
    __syncwarp();
    if (warp < 2) {
        // producer and MMA warps: wait for the epilogue, then free TMEM
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(kOzTmemCols));
        return;
    }
    // ------------------------------------------------------------ epilogue
    const int wq = warp & 3, quarter = (warp - 2) >> 2;
    const uint32_t lanebase = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(quarter * 16);
    double acc64[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc64[i] = 0.0;
    // exact accumulators P_0 .. P_{min(S,5)-1} after every chunk; P_5+ (S >= 6)
    // once, after the last (an accumulator no MMA wrote is not read)
    const int nexact = S < kOzAcc - 1 ? S : kOzAcc - 1;
    for (int c = 0; c < nchunks; ++c) {
        if (ok) ok = mbar_wait(accf, c & 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int nacc = (c == nchunks - 1 && S >= kOzAcc) ? kOzAcc : nexact;
        for (int a = 0; a < nacc; ++a) {
            float v[16];
            tmem_ld16(lanebase + (uint32_t)(a * kOzBN), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc64[i] += (double)v[i];
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(acce);
    }
    const int row = m0 + wq * 32 + lane;
    if (ok && row < M) {
        const int er = ea[row];
        double fat = 0.0, fas = 0.0;
        if (epi == 1) {
            fat = at[row % rows];
            fas = as[row % rows];
        }
        double* dst = C + (size_t)row * ldc;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int col = n0 + quarter * 16 + i;
            if (col < N) {
                double x = ldexp(acc64[i], er + eb[col] - 14);
                if (epi == 1) x = x / (fat - lam[col] * fas);
                dst[col] = x;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}

// One warp per row: exponent ex of the row maximum (|x| < 2^ex), then the
// S balanced base-128 digits of X = round(x 2^(7S - ex)) in integer
// arithmetic: the FP64 mantissa is shifted once to the row's fixed point,
// and the digits are peeled from the least significant end,
// d = ((X + 64) mod 128) - 64, X <- (X - d) / 128; the leading digit keeps
// the rest (|d_0| <= 128).  x 2^-ex = sum_s d_s 2^{-7(s+1)} + r with
// |r| <= 2^{-7S-1}.
__global__ void k_oz_split(const double* __restrict__ X, int rows, int K, int S,
                           __nv_bfloat16* __restrict__ out, int* __restrict__ e) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const double* x = X + (size_t)row * K;
    // row maximum of the biased exponent field
    int emax = 0;
    for (int k = lane; k < K; k += 32) {
        const int be = (int)((__double_as_longlong(x[k]) >> 52) & 0x7FF);
        emax = max(emax, be);
    }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    // |x| < 2^(be - 1022) for a normal x with biased exponent be
    const int ex = emax - 1022;
    if (lane == 0) e[row] = emax == 0 ? 0 : ex;
    for (int k = lane; k < K; k += 32) {
        const long long bits = __double_as_longlong(x[k]);
        const int be = (int)((bits >> 52) & 0x7FF);
        long long v = 0;
        if (be != 0 && emax != 0) {
            const long long mant = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
            // x 2^(7S - ex) = mant 2^(be - 1075 + 7S - ex)
            const int sh = be - 1075 + 7 * S - ex;
            if (sh >= 0)
                v = sh <= 10 ? (mant << sh) : 0;   // S = 8, 9 (|v| < 2^(7S) <= 2^63)
            else if (sh > -60)
                v = (mant + (1ll << (-sh - 1))) >> (-sh);
            if (bits < 0) v = -v;
        }
        for (int s = S - 1; s >= 1; --s) {
            const long long d = ((v + 64) & 127) - 64;
            v = (v - d) >> 7;
            // slice s stored as d 2^{-7s} (exact: a power-of-two scaling)
            out[((size_t)s * rows + row) * K + k] = __float2bfloat16_rn(ldexpf((float)d, -7 * s));
        }
        out[(size_t)row * K + k] = __float2bfloat16_rn((float)v);
    }
}

}  // namespace

size_t ozaki_slice_bytes(int rows, int K, int S) {
    return (size_t)S * rows * K * sizeof(__nv_bfloat16) + (size_t)rows * sizeof(int) + 512;
}

int ozaki_split(cudaStream_t s, const double* X, int rows, int K, int S, void* out, int** e) {
    char* p = static_cast<char*>(out);
    __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(p);
    int* ex = reinterpret_cast<int*>(p + (((size_t)S * rows * K * 2 + 255) / 256) * 256);
    count_launches(1);
    k_oz_split<<<(unsigned)(((size_t)rows * 32 + 255) / 256), 256, 0, s>>>(X, rows, K, S, sl, ex);
    RTE_CUDA_TRY(cudaGetLastError());
    if (e) *e = ex;
    return RTE_OK;
}

int ozaki_gemm(cudaStream_t s, const void* Aslices, const int* ea, int M, const void* Bslices,
               const int* eb, int N, int K, int S, double* C, int ldc, int epi, const double* at,
               const double* as, const double* lam, int rows, int SB) {
    if (M <= 0 || N <= 0 || K <= 0) return RTE_OK;
    if (S < 1 || S > kOzMaxS) return fail(RTE_ERR_ARG, "bad slice count");
    if (SB == 0) SB = S;
    if (SB < S) return fail(RTE_ERR_ARG, "second operand has fewer slices than used");
    CUtensorMap ma, mb;
    RTE_TRY(make_map(&ma, Aslices, false, S * M, K, kOzBM));
    RTE_TRY(make_map(&mb, Bslices, false, SB * N, K, kOzBN));
    // resident B slice sets and A ring slots within the shared-memory limit:
    // two B sets when they fit beside at least two A slots, else one
    constexpr size_t kLimit = 227 * 1024 - 1024 - 16 * 8 - 64;
    auto bytes = [S](int nb, int na) { return (size_t)nb * S * kOzBTile + (size_t)na * kOzATile; };
    int nB = 2, nA = 4;
    while (nA > 2 && bytes(nB, nA) > kLimit) --nA;
    if (bytes(nB, nA) > kLimit) {
        nB = 1;
        nA = 4;
        while (nA > 2 && bytes(nB, nA) > kLimit) --nA;
    }
    // at least half of the SM's shared memory, so that one block (and its 512
    // tensor-memory columns) runs per SM
    const size_t sm = std::max<size_t>(1024 + bytes(nB, nA) + 16 * 8 + 16, 116 * 1024);
    static const bool attr = [] {
        cudaFuncSetAttribute(k_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(227 * 1024));
        return true;
    }();
    (void)attr;
    dim3 grid((N + kOzBN - 1) / kOzBN, (M + kOzBM - 1) / kOzBM);
    count_launches(1);
    k_ozaki<<<grid, kOzThreads, sm, s>>>(ma, mb, M, N, K, S, nA, nB, ea, eb, C, ldc, epi, at, as,
                                         lam, rows);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

}  // namespace rte
