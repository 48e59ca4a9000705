// Arithmetic-pipe probes for the roofline denominators: the sustained rate of
// independent fused multiply-adds in FP32 (scalar FFMA and packed FFMA2) and
// FP64 (DFMA) on this GPU.  Each thread runs CHAINS independent recurrences
// x <- x * a + b (|a| < 1, so values stay normal); the result is stored so the
// work cannot be removed.
#include <cuda_runtime.h>

#include "kirin_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, T a, T b, T *out)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c)
            x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_fma2_probe(int iters, float a, float b, float *out)
{
    float2 x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        x[c] = make_float2((float)threadIdx.x + c, (float)threadIdx.x - c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c)
            x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
        s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// kind 0: FP32 FFMA, 1: packed FP32x2 FFMA2, 2: FP64 DFMA.  *flops_per_s
// counts 2 flops per fused multiply-add lane.  Synchronous; allocates a small
// output buffer.  Errors: EINVAL, ECUDA.
extern "C" int kirin_measure_fma_rate(int32_t device, int32_t kind, double *flops_per_s)
{
    if (!flops_per_s || kind < 0 || kind > 2)
        return KIRIN_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return KIRIN_ECUDA;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int blocks = nsm * 8;
    const int iters = kind == 2 ? 1 << 12 : 1 << 15;
    void *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = KIRIN_ECUDA;
    if (cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * sizeof(double)) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        auto launch = [&]() {
            if (kind == 0)
                k_fma_probe<float><<<blocks, PROBE_THREADS>>>(iters, 0.999f, 1e-3f, (float *)out);
            else if (kind == 1)
                k_fma2_probe<<<blocks, PROBE_THREADS>>>(iters, 0.999f, 1e-3f, (float *)out);
            else
                k_fma_probe<double><<<blocks, PROBE_THREADS>>>(iters, 0.999, 1e-3, (double *)out);
        };
        launch();  // warm-up
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            cudaGetLastError() == cudaSuccess && ms > 0.f) {
            const double lanes = (double)blocks * PROBE_THREADS * CHAINS * iters * (kind == 1 ? 2 : 1);
            *flops_per_s = 2.0 * lanes / (ms * 1e-3);
            rc = KIRIN_OK;
        }
    }
    cudaGetLastError();
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (out)
        cudaFree(out);
    if (prev >= 0)
        cudaSetDevice(prev);
    return rc;
}
