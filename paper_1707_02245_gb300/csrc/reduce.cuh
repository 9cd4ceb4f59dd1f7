// Block-wide FP64 sums used by the duality-gap kernels (deterministic order for a
// fixed launch shape: warp shuffles, then one warp over the per-warp sums).
#pragma once
#include <cuda_runtime.h>

namespace pat {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sums NV doubles per thread over the block; the result is valid in the thread with
// linear index 0.  The block size must be a multiple of 32 and at most 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = warp_sum(v[c]);
    __syncthreads();  // sh may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) sh[c][wid] = v[c];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double x = lane < nw ? sh[c][lane] : 0.0;
            v[c] = warp_sum(x);
        }
    }
}

// s + e = a + b exactly (Knuth's TwoSum); the intrinsics keep the compiler from
// contracting or reordering the roundings
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Warp sum of FP32 values carried as an unevaluated pair hi + lo of FP32 numbers, so the
// sum keeps about 48 significant bits without FP64 arithmetic (GB300's FP64 pipe runs at
// 1/64 of FP32).  Every step adds two pairs with TwoSum and renormalises.  The result, as
// a double, is valid in lane 0.
__device__ __forceinline__ double warp_sum_pair(float v) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        two_sum(s, __fadd_rn(__fadd_rn(lo, l2), e), hi, lo);
    }
    return (double)hi + (double)lo;
}

// Block sums of NV FP32 values per thread: warps reduce with warp_sum_pair, one warp adds
// the per-warp sums in FP64.  The result is valid in the thread with linear index 0; the
// order is fixed for a fixed launch shape.  The block size must be a multiple of 32 and
// at most 1024.
template <int NV>
__device__ __forceinline__ void block_sum_pair(const float (&t)[NV], double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    double w[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) w[c] = warp_sum_pair(t[c]);
    __syncthreads();  // sh may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) sh[c][wid] = w[c];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] = warp_sum(lane < nw ? sh[c][lane] : 0.0);
    }
}

__device__ __forceinline__ double3 block_sum3(double3 a) {
    double v[3] = {a.x, a.y, a.z};
    block_sum<3>(v);
    return make_double3(v[0], v[1], v[2]);
}

}  // namespace pat
