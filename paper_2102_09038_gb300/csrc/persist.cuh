// Helpers for persistent cooperative kernels: a grid barrier whose waits are
// bounded, L2-coherent loads, and workspace carving.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace rte {

struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int n;                       // trace entries written
    unsigned long long* trace;   // optional: %globaltimer after each barrier
    int cap;
    int pad;
    unsigned long long limit_ns; // a wait gives up after this long (0: kWaitLimitNs)
};

// Default limit of a barrier wait: 2 s.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All blocks of the (co-resident) grid meet here.  A wait that runs out sets
// gb->err, and every later barrier returns false at once, so the kernel can
// leave cleanly and the host reads RTE_ERR_TIMEOUT.
__device__ __forceinline__ bool grid_sync(GridBar* gb) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &gb->gen;
        volatile int* verr = &gb->err;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gb->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            // plain polling (a sleep between polls costs more than it saves
            // at these barrier rates); the limit is checked every 256 polls
            const unsigned long long t0 = global_ns();
            const unsigned long long lim = gb->limit_ns ? gb->limit_ns : kWaitLimitNs;
            unsigned spins = 0;
            while (*vgen == g) {
                if ((++spins & 255u) == 0) {
                    if (*verr) break;
                    if (global_ns() - t0 > lim) {
                        atomicExch(&gb->err, 1);
                        break;
                    }
                }
            }
        }
        __threadfence();
        if (blockIdx.x == 0 && gb->trace && gb->n < gb->cap) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            gb->trace[gb->n++] = t;
        }
    }
    __syncthreads();
    return *((volatile int*)&gb->err) == 0;
}

// Loads of data written by other blocks of the same kernel: bypass L1.
__device__ __forceinline__ double ldg2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldg2(const float* p) { return __ldcg(p); }

template <typename T>
inline T* carve(char*& p, size_t n) {
    T* out = reinterpret_cast<T*>(p);
    p += ((n * sizeof(T) + 255) / 256) * 256;
    return out;
}

}  // namespace rte
