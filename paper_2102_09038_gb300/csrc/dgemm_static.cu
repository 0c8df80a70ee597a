// rte_dgemm_split_static: the split FP64 GEMM of rte_dgemm_split with its
// temporaries (digit slices and row exponents of both operands) in one fixed
// device array of this file instead of memory allocated per call.
//
// It serves callers that must not allocate device memory at call time: a
// process whose device memory is already handed out by another allocator (a
// framework's caching pool, a serving memory budget), or a latency-critical
// loop in which an allocation could block on the device or fail.  The paper
// has no counterpart; the arithmetic is that of rte_dgemm_split.
#include <cuda_runtime.h>

#include "../../include/rte.h"
#include "rte_internal.h"
#include "tc_gemm.h"

namespace {

// Every call writes all of the scratch it reads afterwards (slices, then
// exponents), so nothing in it has to start at zero.
static __device__ __align__(256) unsigned char g_split_scratch[RTE_SPLIT_STATIC_SCRATCH_BYTES];

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int rte_dgemm_split_static(const double* A, const double* Bt, double* C, int M, int N,
                                      int K, int slices, void* stream) {
    using namespace rte;
    if (!A || !Bt || !C || M < 0 || N < 0 || K < 0 || slices < 1 || slices > 9)
        return fail(RTE_ERR_ARG, "bad argument");
    // the slices' rows are K BF16 values and each must start on 16 bytes;
    // refused here, before any launch can touch the shared scratch
    if (K % 8 != 0) return fail(RTE_ERR_ARG, "K must be a multiple of 8");
    // a first check in floating point, so that the exact byte count below
    // cannot overflow
    if (2.0 * slices * ((double)M + (double)N) * (double)K > (double)RTE_SPLIT_STATIC_SCRATCH_BYTES)
        return fail(RTE_ERR_ARG, "operands need about " +
                                     std::to_string(2.0 * slices * ((double)M + N) * K) +
                                     " bytes of split-GEMM scratch; the static scratch holds " +
                                     std::to_string((size_t)RTE_SPLIT_STATIC_SCRATCH_BYTES));
    const size_t off_b = round256(ozaki_slice_bytes(M, K, slices));
    const size_t need = off_b + ozaki_slice_bytes(N, K, slices);
    if (need > (size_t)RTE_SPLIT_STATIC_SCRATCH_BYTES)
        return fail(RTE_ERR_ARG, "operands need " + std::to_string(need) +
                                     " bytes of split-GEMM scratch; the static scratch holds " +
                                     std::to_string((size_t)RTE_SPLIT_STATIC_SCRATCH_BYTES));
    if (M == 0 || N == 0) return RTE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) {
        RTE_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * M * N, s));
        RTE_CUDA_TRY(cudaStreamSynchronize(s));
        return RTE_OK;
    }
    // The array's device address on the current device, looked up on every
    // call (a host-side table lookup once the module is loaded), so that a
    // device reset or a new primary context never leaves a stale address.
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_split_scratch);
    if (e != cudaSuccess)
        return fail(RTE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    char* base = static_cast<char*>(p);
    int *ea = nullptr, *eb = nullptr;
    RTE_TRY(ozaki_split(s, A, M, K, slices, base, &ea));
    RTE_TRY(ozaki_split(s, Bt, N, K, slices, base + off_b, &eb));
    RTE_TRY(ozaki_gemm(s, base, ea, M, base + off_b, eb, N, K, slices, C, N, 0, nullptr, 1));
    return tc_gemm_error(s);
}
