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

#include <cstdint>
#include <mutex>

#include "device.h"
#include "rte_internal.h"
#include "tc_gemm.h"

namespace rte {

namespace {

constexpr int kBM = 128;
constexpr int kStages = 4;
constexpr int kRowBytes = 128;   // one K block of a row: 64 bf16 or 32 tf32
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

__device__ int g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) {
            atomicExch(&g_tc_error, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 bytes, 8-row atoms of 1024 bytes
// (stride-dimension offset 1024 B), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;              // leading offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_issue(bool tf32, uint32_t tmem, uint64_t a, uint64_t b,
                                          uint32_t idesc, uint32_t acc) {
    if (tf32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

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

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D K-major tensor map: rows x cols (cols = K contiguous), box = box_rows x
// 128 bytes, 128-byte swizzle, zero fill out of bounds.
int make_map(CUtensorMap* map, const void* base, bool tf32, int rows, int cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return fail(RTE_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const size_t esz = tf32 ? 4 : 2;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || ((size_t)cols * esz) % 16)
        return fail(RTE_ERR_ARG, "tensor-core GEMM operand is not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                    2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(RTE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return RTE_OK;
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
    static bool attr_done = false;
    if (!attr_done) {
        RTE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
        attr_done = true;
    }
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
    const bool wide = g.N > 128;
    if (g.tf32) {
        if (g.out_bf16) return fail(RTE_ERR_ARG, "TF32 GEMM writes FP32");
        return wide ? launch<256, true, float>(s, g) : launch<128, true, float>(s, g);
    }
    if (g.out_bf16)
        return wide ? launch<256, false, __nv_bfloat16>(s, g)
                    : launch<128, false, __nv_bfloat16>(s, g);
    return wide ? launch<256, false, float>(s, g) : launch<128, false, float>(s, g);
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
