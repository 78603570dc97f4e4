// probes.cu -- measurement kernels that give the benchmark its denominators on the GPU it
// runs on (no counterpart in the paper):
//   * the FP64 fused multiply-add rate: every thread of a full grid runs eight
//     independent FMA chains, so the FP64 pipe is the only limit;
//   * the latency of one dependent level of a level-scheduled solve: a consumer group
//     whose threads, level after level, read values other threads wrote in the previous
//     level, combine them, store the result and meet at the group barrier -- the
//     smallest amount of work a level of the streamed level programs can take.
#include <cuda_runtime.h>

#include "ilu2l.h"

namespace ilu2l {

constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double* sink, int iters, double a, double b) {
    double x[kFmaChains];
#pragma unroll
    for (int u = 0; u < kFmaChains; u++) x[u] = 1e-3 * threadIdx.x + u;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kFmaChains; u++) x[u] = fma(x[u], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kFmaChains; u++) s += x[u];
    if (s == -1.0) sink[blockIdx.x] = s;  // never true for a, b > 0: keeps the chains live
}

// One CTA of nt threads (a multiple of 32, <= 256). Level l reads slots t+1, t+3, t+5, t+7
// (mod nt) of buffer l & 1 -- values four other threads stored in level l - 1 -- and stores
// their weighted sum in slot t of the other buffer; then the group barrier (a warp barrier
// for one warp). cycles[0] = clock cycles of `levels` levels.
__global__ void k_level_latency(int nt, int levels, float* sink, long long* cycles) {
    __shared__ float xs[2][256];
    const int t = threadIdx.x;
    if (t >= nt) return;
    xs[0][t] = (float)t;
    xs[1][t] = 0.0f;
    const int i1 = (t + 1) % nt, i3 = (t + 3) % nt, i5 = (t + 5) % nt, i7 = (t + 7) % nt;
    if (nt <= 32)
        __syncwarp();
    else
        asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    const long long c0 = clock64();
    for (int l = 0; l < levels; l++) {
        const float* src = xs[l & 1];
        float* dst = xs[(l + 1) & 1];
        const float v = src[i1] * 0.5f + src[i3] * 0.25f + (src[i5] * 0.125f + src[i7] * 0.0625f);
        dst[t] = v;
        if (nt <= 32)
            __syncwarp();
        else
            asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    }
    const long long c1 = clock64();
    if (t == 0) {
        cycles[0] = c1 - c0;
        sink[0] = xs[levels & 1][0];
    }
}

}  // namespace ilu2l

using namespace ilu2l;

extern "C" {

ilu_status ilu_measure_fp64_peak(void* stream, double* tflops) {
    if (!tflops) return ILU_ERR_ARG;
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* sink = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&sink, sizeof(double) * 8 * sms, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 8 * sms, threads = 256, iters = 1 << 14;
    float ms = 0.0f;
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, threads, 0, st>>>(sink, iters / 8, 1.0 - 1e-12, 1e-12);  // warm-up
        cudaEventRecord(e0, st);
        k_fp64_fma<<<blocks, threads, 0, st>>>(sink, iters, 1.0 - 1e-12, 1e-12);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.0f)
        *tflops = 2.0 * kFmaChains * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    if (sink) cudaFreeAsync(sink, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? ILU_OK : ILU_ERR_CUDA;
}

ilu_status ilu_measure_level_latency(void* stream, int32_t threads, double* cycles_per_level) {
    if (!cycles_per_level || threads < 32 || threads > 256 || threads % 32) return ILU_ERR_ARG;
    *cycles_per_level = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    float* sink = nullptr;
    long long* cyc = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&sink, sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&cyc, sizeof(long long), st);
    const int levels = 4096;
    long long c = 0;
    if (e == cudaSuccess) {
        k_level_latency<<<1, threads, 0, st>>>(threads, levels / 4, sink, cyc);  // warm-up
        k_level_latency<<<1, threads, 0, st>>>(threads, levels, sink, cyc);
        e = cudaMemcpyAsync(&c, cyc, sizeof(long long), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) *cycles_per_level = (double)c / levels;
    if (sink) cudaFreeAsync(sink, st);
    if (cyc) cudaFreeAsync(cyc, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? ILU_OK : ILU_ERR_CUDA;
}

}  // extern "C"
