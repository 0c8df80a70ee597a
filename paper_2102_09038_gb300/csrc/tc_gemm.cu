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
// of two 2^e so that its entries lie in (-1, 1), then cut into S digit
// slices: r <- r * 2^7, d = rint(r), r <- r - d.  The digits are integers
// with |d| <= 128, exact in BF16, and A = 2^e sum_s d_s 2^{-7(s+1)} up to a
// remainder below 2^{-7S-1}.  A product of two digit slices summed over at
// most 1024 terms is an integer below 2^24, so the tensor cores' FP32
// accumulation of it is exact.  The kernel accumulates the slice pairs
// (s, t) with s + t <= S - 1 (the others lie below the truncation level)
// in groups of one weight 2^{-7(s+t+2)} each: a group shares a tensor-memory
// buffer over 512 terms of K, and holds pairs whose digit bounds add up to
// at most 2^15 per term (|d_0 d_0| <= 2^14, |d_0 d_t| <= 2^13, |d_s d_t| <=
// 2^12 for s, t > 0), so its sum stays an integer of magnitude at most
// 2^15 * 512 = 2^24 and the FP32 accumulation is exact (the tensor cores
// truncate when they add, so only exact sums are safe).  A weight with more
// pairs than that takes two groups.  Each buffer is folded into the
// double-float registers with its weight; the row and column scales come
// last.
// ======================================================================
namespace rte {

namespace {

using namespace tc;

constexpr int kOzBM = 128, kOzBN = 128, kOzStages = 6, kOzKChunk = 8;    // 8 x 64 = 512
constexpr int kOzMaxPairs = 64;

// slice pairs ordered by weight w = s + t; pairs of weight w at
// first[w] .. first[w + 1] - 1
struct OzPairs {
    int n, groups;
    unsigned char s[kOzMaxPairs], t[kOzMaxPairs];
    unsigned char first[20];   // group g: pairs first[g] .. first[g + 1] - 1
    unsigned char wgt[20];     // and its weight w = s + t
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 18 warps: warp 0 issues TMA loads, warp 1 issues MMAs, warps 2..17 drain
// the accumulators (warp w reads TMEM lanes 32 (w % 4) .. + 31 and the
// quarter (w - 2) / 4 of the 128 columns), so the producer and the MMA
// issuer never wait on the epilogue's own arrivals.
constexpr int kOzThreads = 576;
constexpr int kOzEpiWarps = 16;
// row pitch (in float2) of the staged (hi, lo) tile: 129 keeps the
// column-wise writes of a warp (one row per lane) free of bank conflicts
constexpr int kOzPitch = kOzBN + 1;
static_assert((size_t)kOzBM * kOzPitch * 8 <= (size_t)kOzStages * (kOzBM + kOzBN) * 128,
              "the staged tile must fit in the pipeline buffers");

// f 2^E as an FP64 bit pattern built with integer operations (sign, the
// exponent rebased and shifted by E, the 23 mantissa bits moved up): exact,
// and no FP64 instruction, which this GPU issues at a small fraction of its
// FP32 and integer rates.  False where f is subnormal, infinite or NaN or
// f 2^E leaves the normal FP64 range.
__device__ __forceinline__ bool f32_scaled_to_f64(float f, int E, double* out) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t mag = b & 0x7FFFFFFFu;
    if (mag == 0) {
        *out = __longlong_as_double((long long)(b & 0x80000000u) << 32);
        return true;
    }
    const int e8 = (int)(mag >> 23);
    const int e11 = e8 + (1023 - 127) + E;
    if (e8 == 0 || e8 == 255 || e11 < 1 || e11 > 2046) return false;
    const uint64_t bits = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)e11 << 52) |
                          ((uint64_t)(mag & 0x7FFFFFu) << 29);
    *out = __longlong_as_double((long long)bits);
    return true;
}

// (hi + lo) 2^E rounded once to FP64: both parts widened and scaled exactly,
// then one FP64 add; out-of-range cases take the FP64 route
__device__ __forceinline__ double df_scaled_to_f64(float hi, float lo, int E) {
    double a, b;
    if (f32_scaled_to_f64(hi, E, &a) && f32_scaled_to_f64(lo, E, &b)) return a + b;
    return ldexp((double)hi + (double)lo, E);
}

// named barrier 1 over the epilogue warps alone (the producer and MMA warps
// wait at the block barrier)
__device__ __forceinline__ void epi_bar_sync() {
    asm volatile("barrier.sync 1, %0;" ::"n"(kOzEpiWarps * 32) : "memory");
}

__global__ void __launch_bounds__(kOzThreads, 1)
k_ozaki(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
        int M, int N, int K, const OzPairs pairs, const int* __restrict__ ea,
        const int* __restrict__ eb, double* __restrict__ C, int ldc, int epi,
        const double* __restrict__ rinv, int rows) {
    constexpr uint32_t kABytes = kOzBM * kRowBytes, kBBytes = kOzBN * kRowBytes;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kOzStages * kABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kOzStages * kBBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kOzStages + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kOzBM, n0 = blockIdx.x * kOzBN;
    const int kblocks = (K + 63) / 64;
    const int nchunks = (kblocks + kOzKChunk - 1) / kOzKChunk;
    const int jobs = pairs.groups * nchunks;   // (weight group, chunk of K)
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kOzStages),
                   accf0 = smem_u32(bars + 2 * kOzStages), acce0 = smem_u32(bars + 2 * kOzStages + 2);
    // slice-pair table in shared memory (a dynamically indexed kernel
    // parameter would live in local memory)
    __shared__ int s_ya[kOzMaxPairs], s_yb[kOzMaxPairs];
    __shared__ int s_first[20], s_wgt[20];
    __shared__ int s_fail;   // set by an epilogue thread whose wait timed out
    for (int p = threadIdx.x; p < pairs.n; p += blockDim.x) {
        s_ya[p] = pairs.s[p] * M + m0;
        s_yb[p] = pairs.t[p] * N + n0;
    }
    for (int g = threadIdx.x; g <= pairs.groups; g += blockDim.x) {
        s_first[g] = pairs.first[g];
        s_wgt[g] = pairs.wgt[g];
    }
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < kOzStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, kOzEpiWarps);   // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // --------------------------------------------- TMA producer
        int g = 0;
        for (int j = 0; j < jobs && ok; ++j) {
            const int grp = j / nchunks, ch = j % nchunks;
            const int p0 = s_first[grp], p1 = s_first[grp + 1];
            const int kb1 = min(kblocks, (ch + 1) * kOzKChunk);
            for (int kb = ch * kOzKChunk; kb < kb1 && ok; ++kb)
                for (int p = p0; p < p1; ++p, ++g) {
                    const int st = g % kOzStages;
                    const uint32_t ph = (g / kOzStages) & 1;
                    if (!mbar_wait(empty0 + 8 * st, ph ^ 1)) { ok = false; break; }
                    mbar_expect_tx(full0 + 8 * st, kABytes + kBBytes);
                    tma_load_2d(smem_u32(sA + st * kABytes), &mapA, full0 + 8 * st, kb * 64, s_ya[p]);
                    tma_load_2d(smem_u32(sB + st * kBBytes), &mapB, full0 + 8 * st, kb * 64, s_yb[p]);
                }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------- MMA issuer
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(kOzBN >> 3) << 17) | ((uint32_t)(kOzBM >> 4) << 24);
        int g = 0;
        for (int j = 0; j < jobs && ok; ++j) {
            const int b = j & 1;
            const uint32_t bph = (j >> 1) & 1;
            if (!mbar_wait(acce0 + 8 * b, bph ^ 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dtm = tmem + (uint32_t)(b * kOzBN);
            const int grp = j / nchunks, ch = j % nchunks;
            const int np = s_first[grp + 1] - s_first[grp];
            const int kb0 = ch * kOzKChunk, kb1 = min(kblocks, kb0 + kOzKChunk);
            bool first = true;   // the job's first MMA overwrites the buffer
            for (int kb = kb0; kb < kb1 && ok; ++kb)
                for (int p = 0; p < np; ++p, ++g) {
                    const int st = g % kOzStages;
                    const uint32_t ph = (g / kOzStages) & 1;
                    if (!mbar_wait(full0 + 8 * st, ph)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + st * kABytes), b0 = smem_u32(sB + st * kBBytes);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_issue(false, dtm, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk),
                                  idesc, (!first || kk > 0) ? 1u : 0u);
                    first = false;
                    mma_commit(empty0 + 8 * st);
                }
            mma_commit(accf0 + 8 * b);
        }
    }
    __syncwarp();
    if (warp < 2) {
        // producer and MMA warps: wait for the epilogue, then free TMEM
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(256));
        return;
    }
    // ------------------------------------------------------------ epilogue
    const int wq = warp & 3, quarter = (warp - 2) >> 2;
    // Double-float accumulators (hi + lo, about 48 significant bits): every
    // job adds v 2^-7(s+t+2) with v an integer below 2^24, exact in FP32; the
    // two-sum keeps the rounding error of each addition in lo.  FP32 runs at
    // many times the FP64 rate of this GPU.
    float hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        hi[i] = 0.f;
        lo[i] = 0.f;
    }
    for (int j = 0; j < jobs; ++j) {
        const int b = j & 1;
        const uint32_t bph = (j >> 1) & 1;
        if (ok) ok = mbar_wait(accf0 + 8 * b, bph);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float w = ldexpf(1.0f, -7 * (s_wgt[j / nchunks] + 2));   // the group's weight
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(b * kOzBN + quarter * 32 + c0), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float x = v[i] * w;                 // exact
                const float sum = __fadd_rn(hi[c0 + i], x);
                const float bb = __fsub_rn(sum, hi[c0 + i]);
                const float err = __fadd_rn(__fsub_rn(hi[c0 + i], __fsub_rn(sum, bb)),
                                            __fsub_rn(x, bb));
                hi[c0 + i] = sum;
                lo[c0 + i] = __fadd_rn(lo[c0 + i], err);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * b);
    }
    // Finish through shared memory: every thread parks its (hi, lo) pairs
    // (one row, 32 columns) in the pipeline buffers, which the last MMA has
    // finished reading; then each warp converts and stores whole rows, so
    // the loads of eb, of the reciprocal table and the FP64 stores are
    // coalesced.  The block writes all or nothing: if any epilogue wait
    // timed out (an MMA may then still be reading the buffers), none.
    if (!ok) s_fail = 1;
    epi_bar_sync();
    const bool write = s_fail == 0;
    float2* stage = reinterpret_cast<float2*>(smem);   // [kOzBM][kOzPitch]
    if (write) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        float2* mine = stage + (wq * 32 + lane) * kOzPitch + quarter * 32;
#pragma unroll
        for (int i = 0; i < 32; ++i) mine[i] = make_float2(hi[i], lo[i]);
    }
    epi_bar_sync();
    if (write) {
        for (int rl = warp - 2; rl < kOzBM; rl += kOzEpiWarps) {
            const int row = m0 + rl;
            if (row >= M) break;
            const int er = ea[row];
            const double* rr = epi == 1 ? rinv + (size_t)(row % rows) * N : nullptr;
            double* dst = C + (size_t)row * ldc;
#pragma unroll
            for (int j = 0; j < kOzBN / 32; ++j) {
                const int c = lane + 32 * j, col = n0 + c;
                if (col < N) {
                    const float2 v = stage[rl * kOzPitch + c];
                    double x = df_scaled_to_f64(v.x, v.y, er + eb[col]);
                    if (epi == 1) x *= rr[col];
                    dst[col] = x;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}

// 1 / (at[r] - lam[c] as[r]) for r < rows, c < N, row-major: the diagonal of
// (M^- - K^-)^{-1} in the eigenbasis per cell, built once so that the split
// GEMM's epilogue multiplies instead of dividing in FP64
__global__ void k_oz_recip(int rows, int N, const double* __restrict__ at,
                           const double* __restrict__ as, const double* __restrict__ lam,
                           double* __restrict__ out) {
    const size_t total = (size_t)rows * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / N), c = (int)(e % N);
        out[e] = 1.0 / (at[r] - lam[c] * as[r]);
    }
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
            out[((size_t)s * rows + row) * K + k] = __float2bfloat16_rn((float)(int)d);
        }
        out[(size_t)row * K + k] = __float2bfloat16_rn((float)(int)v);
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

int ozaki_recip_table(cudaStream_t s, const double* at, const double* as, const double* lam,
                      int rows, int N, double* out) {
    if (rows <= 0 || N <= 0) return RTE_OK;
    count_launches(1);
    const size_t total = (size_t)rows * N;
    const unsigned blocks =
        (unsigned)std::min<size_t>((total + 255) / 256, (size_t)device_sm_count() * 8);
    k_oz_recip<<<blocks, 256, 0, s>>>(rows, N, at, as, lam, out);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int ozaki_gemm(cudaStream_t s, const void* Aslices, const int* ea, int M, const void* Bslices,
               const int* eb, int N, int K, int S, double* C, int ldc, int epi,
               const double* rinv, int rows, int SB) {
    if (M <= 0 || N <= 0 || K <= 0) return RTE_OK;
    if (epi == 1 && (!rinv || rows <= 0)) return fail(RTE_ERR_ARG, "epilogue 1 needs its table");
    if (S < 1 || S > 9 || S * (S + 1) / 2 > kOzMaxPairs) return fail(RTE_ERR_ARG, "bad slice count");
    if (SB == 0) SB = S;
    if (SB < S) return fail(RTE_ERR_ARG, "second operand has fewer slices than used");
    // pairs by weight, cut into groups whose per-term digit bounds add up to
    // at most 2^15 (see the comment above k_ozaki)
    OzPairs pairs{};
    for (int w = 0; w < S; ++w) {
        int cost = 1 << 16;   // forces a new group
        for (int a = 0; a <= w; ++a) {
            const int b = w - a;
            const int c = (a == 0 && b == 0) ? 1 << 14 : (a == 0 || b == 0) ? 1 << 13 : 1 << 12;
            if (cost + c > (1 << 15)) {
                pairs.first[pairs.groups] = (unsigned char)pairs.n;
                pairs.wgt[pairs.groups] = (unsigned char)w;
                ++pairs.groups;
                cost = 0;
            }
            cost += c;
            pairs.s[pairs.n] = (unsigned char)a;
            pairs.t[pairs.n] = (unsigned char)b;
            ++pairs.n;
        }
    }
    pairs.first[pairs.groups] = (unsigned char)pairs.n;
    CUtensorMap ma, mb;
    RTE_TRY(make_map(&ma, Aslices, false, S * M, K, kOzBM));
    RTE_TRY(make_map(&mb, Bslices, false, SB * N, K, kOzBN));
    const size_t sm = 1024 + (size_t)kOzStages * (kOzBM + kOzBN) * kRowBytes +
                      (2 * kOzStages + 4) * 8 + 16;
    RTE_CUDA_TRY(cudaFuncSetAttribute(k_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
    dim3 grid((N + kOzBN - 1) / kOzBN, (M + kOzBM - 1) / kOzBM);
    count_launches(1);
    k_ozaki<<<grid, kOzThreads, sm, s>>>(ma, mb, M, N, K, pairs, ea, eb, C, ldc, epi, rinv,
                                         rows);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

}  // namespace rte
