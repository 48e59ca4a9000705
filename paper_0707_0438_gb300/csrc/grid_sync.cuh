// Waits between the CTAs of one cooperative launch (all CTAs resident): an
// arrival counter that only grows, release adds, relaxed polls ended by one
// acquire load, every wait bounded; and the proxy fence that orders global
// writes before bulk copies read them.
#pragma once

#include <cuda_runtime.h>

#include "kirin_internal.cuh"
#include "tma.cuh"

namespace kirin {
namespace {

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Order this thread's earlier global accesses before later bulk copies, which read global memory
// through the async proxy.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// This CTA's writes of the phase are done (the CTA barrier orders every thread's stores before
// thread 0's release): one more arrival.
__device__ __forceinline__ void arrive(unsigned *arrivals)
{
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(arrivals) : "memory");
}

// Wait until the counter reaches target (compared modulo 2^32): thread 0 polls relaxed for at most
// limit_ns, then one acquire load orders what the arrivals published.  False (and ERR_TIMEOUT)
// when it never came; every thread of the CTA calls it and gets the same answer.
__device__ __forceinline__ bool wait_arrivals(const unsigned *arrivals, unsigned target, unsigned *err,
                                              unsigned long long limit_ns = WAIT_LIMIT_NS)
{
    bool ok = true;
    if (threadIdx.x == 0) {
        if ((int)(ld_relaxed_gpu(arrivals) - target) < 0) {
            const unsigned long long t0 = global_ns();
            while ((int)(ld_relaxed_gpu(arrivals) - target) < 0)
                if (global_ns() - t0 > limit_ns) {
                    ok = false;
                    break;
                }
        }
        if (ok)
            ok = (int)(ld_acquire_gpu(arrivals) - target) >= 0;  // it only grows: true, and now ordered
    }
    const bool failed = __syncthreads_or(!ok);
    if (failed && threadIdx.x == 0)
        atomicOr(err, ERR_TIMEOUT);
    return !failed;
}

}  // namespace
}  // namespace kirin
