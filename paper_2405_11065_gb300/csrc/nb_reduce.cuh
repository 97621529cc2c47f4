// Deterministic reductions: every sum is taken in a fixed order that depends
// only on the launch shape, never on scheduling, so repeated calls give
// bit-identical results.
#pragma once

#include "nb_internal.h"

namespace nb {

// Sum of v over the block, returned on thread 0 (warp shuffles in a fixed
// tree, then the warp sums in index order).
__device__ __forceinline__ double block_sum(double v, double *sred)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? sred[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

// Sum of part[0..cnt) by one block: each thread sums a fixed strided subset
// in increasing index, then block_sum.
__device__ __forceinline__ double sum_partials(const double *part, int cnt, double *sred)
{
    double v = 0.0;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) v += part[t];
    return block_sum(v, sred);
}

// Per-thread accumulation of a dot product with FP64 accuracy.  For double
// terms it is a plain FP64 sum.  For float terms it is a compensated FP32 sum
// (Knuth's TwoSum: s + c carries the rounding error of every addition),
// converted to FP64 once per thread: FP64-level accuracy for the FP32
// products without an FP64 instruction per term, which matters on a GPU whose
// FP64 rate is a small fraction of its FP32 rate.
template <typename T>
struct DotAcc;

template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct DotAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;
        const float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

constexpr int kVecThreads = 256;

inline int vec_grid(const nb_ctx *ctx, int64_t n)
{
    int64_t g = (n + kVecThreads - 1) / kVecThreads;
    int64_t cap = (int64_t)ctx->sm_count * 4;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace nb
