// Bounded grid barrier of the library's cooperative kernels (the persistent solvers,
// the single-launch sort): device code only, included by the .cu files that need it.
#pragma once

#include <cuda_runtime.h>

namespace bem {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of the persistent solvers: one arrival counter that only grows
// (thread 0 of each CTA adds 1 with release semantics, then polls with acquire
// loads until the counter reaches G times the number of barriers passed), so a
// barrier costs one fire-and-forget add and the polls.  The wait is bounded in
// time: after limit_ns (%globaltimer) the CTA raises err and the call returns
// false, so the kernel ends with an error status instead of hanging; a CTA that
// sees err raised by another one gives up as well.  absent: this CTA leaves at the
// barrier without arriving (failure-detection tests: the others must time out).
constexpr long long kBarrierLimitNs = 2000000000ll;  // default wait limit: 2 s
struct GridBar {
    unsigned *cnt;
    int *err;
    unsigned target;
    long long limit_ns;
    bool absent;
};

__device__ __forceinline__ bool grid_barrier(GridBar &b, int G)
{
    __shared__ int s_ok;
    __syncthreads();
    b.target += (unsigned)G;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (b.absent) {
            ok = 0;
        } else {
            red_release_add_u32(b.cnt, 1u);
            unsigned long long t0 = 0;
            for (unsigned polls = 1; (int)(ld_acquire_u32(b.cnt) - b.target) < 0; ++polls) {
                if ((polls & 31) == 0) {
                    const unsigned long long t = global_ns();
                    if (t0 == 0) {
                        t0 = t;
                    } else if ((long long)(t - t0) > b.limit_ns || *(volatile int *)b.err) {
                        atomicExch(b.err, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            if (ok && *(volatile int *)b.err) ok = 0;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace bem
