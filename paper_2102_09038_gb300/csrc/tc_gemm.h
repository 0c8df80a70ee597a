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
    int bn = 0;         // tile width 128 or 256; 0: 256 when N > 128
};

int tc_gemm(cudaStream_t s, const TcGemmArgs& g);
// Reads and clears the device-side timeout flag of the GEMM pipelines.
int tc_gemm_error(cudaStream_t s);
// Limit of one mbarrier wait of the GEMM pipelines on the current device.
int tc_set_wait_cycles(long long cycles);

// FP64-accurate GEMM from exact BF16 products of digit slices (tc_gemm.cu).
// ozaki_split: S slices of the rows of X (rows x K, FP64) into `out`
// (ozaki_slice_bytes), *e = per-row exponents inside `out`.
size_t ozaki_slice_bytes(int rows, int K, int S);
int ozaki_split(cudaStream_t s, const double* X, int rows, int K, int S, void* out, int** e);
// C (M x N, FP64) = A B^T from the slices of A (M x K) and of Bt (N x K);
// epi 1 multiplies entry (r, c) by rinv[(r % rows) N + c] (ozaki_recip_table).
// K <= any; exact accumulation within chunks of 512.  S digit slices are
// used; Bslices holds SB >= S (its slices s < S are the leading digits of
// the same expansion, so the first S of them are an S-digit truncation);
// SB = 0 means SB = S.
int ozaki_gemm(cudaStream_t s, const void* Aslices, const int* ea, int M, const void* Bslices,
               const int* eb, int N, int K, int S, double* C, int ldc, int epi,
               const double* rinv, int rows, int SB = 0);
// out[r N + c] = 1 / (at[r] - lam[c] as[r]) for r < rows, c < N (rows x N FP64)
int ozaki_recip_table(cudaStream_t s, const double* at, const double* as, const double* lam,
                      int rows, int N, double* out);

}  // namespace rte
