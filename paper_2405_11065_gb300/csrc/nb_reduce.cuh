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

// Sum of part[0..cnt), called by the whole block, returned on thread 0.  Up
// to 2048 partials warp 0 alone sums them (lane l: part[l], part[l + 32], ...
// in increasing index, then a fixed shuffle tree), which keeps the FP64 work
// of the block to one warp; beyond that every thread sums a strided subset,
// then block_sum.
__device__ __forceinline__ double sum_partials(const double *part, int cnt, double *sred)
{
    if (cnt <= 2048) {
        double v = 0.0;
        if (threadIdx.x < 32) {
            for (int t = threadIdx.x; t < cnt; t += 32) v += part[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        }
        return v;
    }
    __threadfence();  // every thread reads partials of other blocks
    double v = 0.0;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) v += part[t];
    return block_sum(v, sred);
}

// Two sums of partials (part[0..cnt) and part2[0..cnt)) with their loads in
// one pass; the same order and results as two calls of sum_partials.
__device__ __forceinline__ void sum_partials2(const double *part, const double *part2, int cnt,
                                              double *sred, double &s1, double &s2)
{
    if (cnt <= 2048) {
        double v = 0.0, u = 0.0;
        if (threadIdx.x < 32) {
            for (int t = threadIdx.x; t < cnt; t += 32) {
                v += part[t];
                u += part2[t];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_down_sync(0xffffffffu, v, o);
                u += __shfl_down_sync(0xffffffffu, u, o);
            }
        }
        s1 = v;
        s2 = u;
        return;
    }
    s1 = sum_partials(part, cnt, sred);
    s2 = sum_partials(part2, cnt, sred);
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

// Sum over the block of the threads' accumulators, returned on thread 0.  For
// the compensated FP32 form: the (s, c) pairs are merged in FP32 within each warp (TwoSum of
// the leading parts, the error added to the compensations, in a fixed
// shuffle tree), each warp's pair is converted to FP64 once, and warp 0 sums
// the warp totals in index order.  FP64-level accuracy without FP64
// arithmetic per thread: on a GPU whose FP64 rate is a small fraction of its
// FP32 rate, a plain FP64 tree over hundreds of threads costs microseconds.
__device__ __forceinline__ double block_sum_acc(const DotAcc<float> &acc, double *sred)
{
    float s = acc.s, c = acc.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_down_sync(0xffffffffu, s, o);
        const float co = __shfl_down_sync(0xffffffffu, c, o);
        const float t = s + so;
        const float bp = t - s;
        c += co + ((s - (t - bp)) + (so - bp));
        s = t;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[wid] = (double)s + (double)c;
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

__device__ __forceinline__ double block_sum_acc(const DotAcc<double> &acc, double *sred)
{
    return block_sum(acc.s, sred);
}

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
