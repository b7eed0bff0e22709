// Calibration of the roofline denominators of the arithmetic-bound kernels on the running GPU: the
// FP32 fused multiply-add rate of the paired instruction the blend uses (FFMA2, two lanes of fp32
// per instruction) and the rate of the exp2 approximation (MUFU), each measured by chain kernels
// that fill every SM with independent dependency chains.
#include <algorithm>

#include "internal.cuh"

namespace h3dgs {
namespace {

constexpr int CAL_BLOCK = 256;
constexpr int CAL_CHAINS = 8;   // independent chains per thread (hides the instruction latency)

__global__ void __launch_bounds__(CAL_BLOCK) fma_chain_kernel(int iters, float seed, float* __restrict__ sink) {
    float2 a[CAL_CHAINS];
#pragma unroll
    for (int k = 0; k < CAL_CHAINS; ++k) a[k] = make_float2(seed + threadIdx.x + k, seed - k);
    const float2 m = make_float2(0.9999f, 0.9998f), c = make_float2(1.0e-4f, 2.0e-4f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CAL_CHAINS; ++k) a[k] = __ffma2_rn(a[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CAL_CHAINS; ++k) s += a[k].x + a[k].y;
    if (s == seed) sink[blockIdx.x] = s;   // keeps the chains live; never true for the seeds used
}

__global__ void __launch_bounds__(CAL_BLOCK) ex2_chain_kernel(int iters, float seed, float* __restrict__ sink) {
    float a[CAL_CHAINS];
#pragma unroll
    for (int k = 0; k < CAL_CHAINS; ++k) a[k] = -0.001f * (threadIdx.x + k) - seed;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CAL_CHAINS; ++k) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
            a[k] = -y;   // stays in (-1, 0]: exp2 of it stays in (0.5, 1]
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CAL_CHAINS; ++k) s += a[k];
    if (s == seed) sink[blockIdx.x] = s;
}

}  // namespace

cudaError_t measure_peaks(int num_sms, float* fp32_tflops, float* ex2_gops, cudaStream_t s) {
    const int blocks = num_sms * 8;
    float* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * blocks);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int fma_iters = 1 << 14, ex2_iters = 1 << 12;
    float best_fma = 1e30f, best_ex2 = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first repetition warms up; the fastest counts
        float ms = 0.0f;
        cudaEventRecord(e0, s);
        fma_chain_kernel<<<blocks, CAL_BLOCK, 0, s>>>(fma_iters, 3.0f, sink);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best_fma = std::min(best_fma, ms);
        cudaEventRecord(e0, s);
        ex2_chain_kernel<<<blocks, CAL_BLOCK, 0, s>>>(ex2_iters, 3.0f, sink);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best_ex2 = std::min(best_ex2, ms);
    }
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    const double threads = (double)blocks * CAL_BLOCK;
    // one FFMA2 = two fused multiply-adds = 4 flops
    *fp32_tflops = (float)(threads * fma_iters * CAL_CHAINS * 4.0 / (best_fma * 1e-3) / 1e12);
    *ex2_gops = (float)(threads * ex2_iters * CAL_CHAINS / (best_ex2 * 1e-3) / 1e9);
    return e;
}

}  // namespace h3dgs
