// Throughput of the two pipes that bound the operators: FP32 fused multiply-add and the MUFU
// exponential (ex2.approx), measured on the device with CUDA events.  The operators are
// instruction-issue bound FP32/MUFU work, so their roofline needs these rates next to the
// figures derived from unit counts and the clock.
#include <cuda_runtime.h>

#include "gpair_internal.cuh"
#include "../../include/gpair.h"

namespace gp {
namespace {

constexpr int PEAK_CHAINS = 8;       // independent dependency chains per thread
constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) ffma_peak_kernel(int iters, float b, float c, float* sink) {
    float x[PEAK_CHAINS];
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q) x[q] = (float)(threadIdx.x + q) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < PEAK_CHAINS; ++q) x[q] = fmaf(x[q], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q) s += x[q];
    if (s == 1234.5f) sink[blockIdx.x] = s;     // keeps the chains alive; never true for b, c below
}

__global__ void __launch_bounds__(PEAK_THREADS) ex2_peak_kernel(int iters, float* sink) {
    float x[PEAK_CHAINS];
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q) x[q] = -(float)(threadIdx.x + q) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < PEAK_CHAINS; ++q) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[q]));
                x[q] = -y;                        // stays in [-1, -0.5]
            }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; ++q) s += x[q];
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace gp

extern "C" gpair_status gpair_pipe_peak(int pipe, int reps, double* lane_ops_per_s, void* stream) {
    using namespace gp;
    if ((pipe != GPAIR_PIPE_FP32 && pipe != GPAIR_PIPE_MUFU) || reps < 1 || reps > 1000 || !lane_ops_per_s)
        return GPAIR_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GPAIR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 8;                       // 8 CTAs of 8 warps per SM: every scheduler kept busy
    const int iters = pipe == GPAIR_PIPE_FP32 ? 8192 : 2048;
    float* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return GPAIR_ERR_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gpair_status s = GPAIR_OK;
    float ms = 0.f;
    auto launch = [&]() {
        if (pipe == GPAIR_PIPE_FP32) ffma_peak_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.999f, 1e-4f, sink);
        else ex2_peak_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, sink);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        s = GPAIR_ERR_CUDA;
    } else {
        launch();                                     // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
            s = GPAIR_ERR_CUDA;
    }
    if (s == GPAIR_OK) {
        const double ops = (double)reps * blocks * PEAK_THREADS * (double)iters * 8.0 * PEAK_CHAINS;
        *lane_ops_per_s = ops / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return s;
}
