// Tensor-core (tcgen05) GEMM launcher.
#pragma once

#include <cuda_runtime.h>

namespace rte {

struct TcGemmArgs {
    const void* A;      // M x K, row-major (K contiguous), BF16 or FP32 (TF32)
    const void* Bt;     // N x K, row-major (K contiguous), same type as A
    void* C;            // M x N output, leading dimension ldc, FP32 or BF16
    int M, N, K, ldc;
    int epi;            // 0: C = A B^T (+ beta C); 1: divide by (at - lam as)
    const float* at;    // per-row factors (row % rows), epi 1
    const float* as;
    const float* lam;   // per-column eigenvalues, epi 1
    int rows;
    float beta;
    bool tf32;          // operands FP32 read as TF32 (else BF16)
    bool out_bf16;      // write C as BF16 (else FP32)
};

int tc_gemm(cudaStream_t s, const TcGemmArgs& g);
// Reads and clears the device-side timeout flag of the GEMM pipeline.
int tc_gemm_error(cudaStream_t s);

}  // namespace rte
