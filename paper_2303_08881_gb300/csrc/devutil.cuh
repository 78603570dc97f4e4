// devutil.cuh -- deterministic reductions and small helpers shared by the kernels.
// All reductions use a fixed thread-to-data mapping and a fixed combination order, so a
// result depends only on the data and the launch shape, never on timing or on which
// other work shares the GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ilu2l {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;  // valid in lane 0
}

// Sum of NV values per thread over the block; result (valid in every thread) in v[].
// scratch: at least 32 * NV doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int u = 0; u < NV; u++) v[u] = warp_sum(v[u]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < NV; u++) scratch[warp * NV + u] = v[u];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NV; u++) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += scratch[w * NV + u];
        v[u] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double block_sum(double v, double* scratch) {
    double a[1] = {v};
    block_sum_n<1>(a, scratch);
    return a[0];
}

// The same sums in an accumulator type A (float for the FP32 preconditioner: GB300 runs
// FP64 arithmetic at a small fraction of the FP32 rate). scratch: 32 * NV values of A.
template <class A>
__device__ __forceinline__ A warp_sum_t(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;  // valid in lane 0
}

template <class A, int NV>
__device__ __forceinline__ void block_sum_nt(A (&v)[NV], A* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int u = 0; u < NV; u++) v[u] = warp_sum_t(v[u]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < NV; u++) scratch[warp * NV + u] = v[u];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NV; u++) {
        A s = (A)0;
        for (int w = 0; w < nw; w++) s += scratch[w * NV + u];
        v[u] = s;
    }
    __syncthreads();
}

template <class A>
__device__ __forceinline__ A block_sum_t(A v, A* scratch) {
    A a[1] = {v};
    block_sum_nt<A, 1>(a, scratch);
    return a[0];
}

// Sum of a[0..m) by one warp: lane l adds a[l], a[l+32], ... in order, then a butterfly
// (xor) exchange combines the lanes. Both partners of every exchange add the same two
// values, so all lanes -- and every warp or CTA that calls this on the same data -- end
// with the same bits. All 32 lanes of the warp must call it.
__device__ __forceinline__ double warp_allsum_ldcg(const double* a, int m) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += __ldcg(a + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return s;
}

// Fixed-order sum of a[0..m) (each thread obtains the same value).
__device__ __forceinline__ double seq_sum_ldcg(const double* a, int m) {
    double s = 0.0;
    for (int i = 0; i < m; i++) s += __ldcg(a + i);
    return s;
}

// fused multiply-add rounded once, never re-associated by the compiler
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class T>
__device__ __forceinline__ T to_t(double v) {
    return (T)v;
}

}  // namespace ilu2l
