// Reduction helpers shared by the vector kernels and the fused residual step:
// warp / block sums in FP64 and the compensated FP32 per-thread accumulator.
#pragma once

#include "internal.h"

namespace tlr {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of v (blockDim.x a multiple of 32, at most 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Per-thread partial sum: FP32 terms accumulated with Knuth's two-sum
// compensation (error-free transformation), so a thread's partial is as good
// as an FP64 sum of its FP32 terms while costing FP32 adds only; partials are
// then combined in FP64.  Elementwise FP64 multiply-adds would cost far more on
// this part than the memory traffic they sit on.
struct Acc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ double val() const { return (double)s + (double)c; }
};

}  // namespace tlr
