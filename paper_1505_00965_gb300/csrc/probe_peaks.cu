// probe_peaks.cu -- throughput probes of the units the level kernels use (a standalone program,
// built and run by `python -m paper_1505_00965_gb300.peaks`):
//   mufu    the four hardware approximations of Box--Muller (lg2, sqrt, sin, cos), 8 independent
//           chains per thread
//   ffma    FP32 fused multiply-adds, 8 independent chains per thread
//   dfma    FP64 fused multiply-adds, 8 independent chains per thread (the pipe of the FP64 paths)
//   philox  Philox4x32-10 blocks (the generator of the level kernels, key schedule in registers)
// Each kernel runs `iters` rounds per thread on a grid of `blocks_per_sm` x SMs x 256 threads and
// writes one word per thread (the buffer has exactly that many words), so that nothing is
// optimised away.  Prints one JSON line: operations per second and per SM per clock (max clock).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "rng.cuh"

using namespace mlmcgb;

__global__ void __launch_bounds__(256) mufu_probe(float *out, int iters)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.5f + 1e-3f * (float)((tid + k) & 255);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; k += 4) {
            v[k] = lg2_approx(v[k] + 1.0f);
            v[k + 1] = sqrt_approx(v[k + 1] + 1.0f);
            v[k + 2] = sin_approx(v[k + 2]);
            v[k + 3] = cos_approx(v[k + 3]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    out[tid] = s;
}

__global__ void __launch_bounds__(256) ffma_probe(float *out, int iters)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 1e-3f * (float)((tid + k) & 255);
    const float a = 0.999f, b = 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = fmaf(v[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    out[tid] = s;
}

__global__ void __launch_bounds__(256) dfma_probe(float *out, int iters)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 1e-3 * (double)((tid + k) & 255);
    const double a = 0.999, b = 1e-4;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    out[tid] = (float)s;
}

__global__ void __launch_bounds__(256) philox_probe(float *out, int iters, uint32_t k0, uint32_t k1)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
        const uint4 x = philox4x32_10(make_uint4((uint32_t)i, tid, 0u, 7u), k0, k1);
        acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
    out[tid] = (float)(acc & 0xFFFF);
}

int main()
{
    int dev = 0, sms = 0, clock_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
    const int threads = 256, blocks = sms * 8;
    const size_t words = (size_t)blocks * threads;
    float *out = nullptr;
    if (cudaMalloc(&out, words * sizeof(float)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 4096;
    double rate[4] = {0, 0, 0, 0};
    for (int which = 0; which < 4; ++which) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0);
            if (which == 0) mufu_probe<<<blocks, threads>>>(out, iters);
            else if (which == 1) ffma_probe<<<blocks, threads>>>(out, iters);
            else if (which == 2) philox_probe<<<blocks, threads>>>(out, iters / 4, 1u, 2u);
            else dfma_probe<<<blocks, threads>>>(out, iters / 16);  // FP64 runs far slower than FP32
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;  // the first launch warms up
        }
        const double ops_per_thread = which == 2 ? (double)(iters / 4) : which == 3 ? 8.0 * (iters / 16) : 8.0 * iters;
        rate[which] = ops_per_thread * (double)words / (best * 1e-3);
    }
    const cudaError_t err = cudaGetLastError();
    const double per_sm_clk = 1.0 / ((double)sms * clock_khz * 1e3);
    printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"mufu_per_s\": %.4e, \"mufu_per_sm_per_clk\": %.2f, "
           "\"ffma_per_s\": %.4e, \"ffma_per_sm_per_clk\": %.2f, \"philox_blocks_per_s\": %.4e, "
           "\"dfma_per_s\": %.4e, \"dfma_per_sm_per_clk\": %.3f, \"status\": \"%s\"}\n",
           sms, clock_khz / 1e3, rate[0], rate[0] * per_sm_clk, rate[1], rate[1] * per_sm_clk, rate[2], rate[3],
           rate[3] * per_sm_clk, cudaGetErrorString(err));
    cudaFree(out);
    return err == cudaSuccess ? 0 : 1;
}
