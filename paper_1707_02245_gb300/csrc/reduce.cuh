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

__device__ __forceinline__ double3 block_sum3(double3 a) {
    double v[3] = {a.x, a.y, a.z};
    block_sum<3>(v);
    return make_double3(v[0], v[1], v[2]);
}

}  // namespace pat
