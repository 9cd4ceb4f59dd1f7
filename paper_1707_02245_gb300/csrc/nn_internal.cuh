// Internal declarations of the learned warm start's network kernels (bfloat16 tensor-core
// convolutions, resampling, masks, loss, Adam).  Shared by conv.cu and unet.cu only; the
// public boundary is pat_unet.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pat {
namespace nn {

using bf16 = __nv_bfloat16;

// Channels-last activation view: element (pixel p, channel c) at ptr[p * ps + c], with
// pixels numbered ((n * H) + iy) * W + ix.  ps >= channels; channel slices of a wider
// buffer (the decoder's concatenation) are views with an offset pointer.
struct View {
    bf16* p;
    int ps;
};

// y = conv3x3(x, w) + bias (optional ReLU).  w is [cout][9][cin] bf16; out_f32 selects an
// FP32 output (float* in y_f32) instead of bf16 (View y).
int conv3x3_fwd(const View& x, int B, int H, int W, int cin, const bf16* w, const float* bias, int cout,
                bool relu, const View& y, float* y_f32, int y_f32_ps, cudaStream_t st);

// dw[o][tap][c] = sum_p dz[p][o] x[p + tap][c] and db[o] = sum_p dz[p][o] (FP32,
// overwritten; db may be null).  part must hold wgrad_partial_floats(...) floats.
size_t wgrad_partial_floats(int B, int H, int W, int cin, int cout);
int conv3x3_wgrad(const View& x, const View& dz, int B, int H, int W, int cin, int cout, float* dw, float* db,
                  float* part, cudaStream_t st);

// wflip[c][tap][o] = w[o][8 - tap][c]: the weights of the transposed convolution that gives
// dL/dx from dL/dy.
int flip_weights(const bf16* w, int cout, int cin, bf16* wflip, cudaStream_t st);

// bounded waits of the tensor-memory convolutions that ran out since the library loaded
// (~0u if it cannot be read)
unsigned wait_timeouts();

}  // namespace nn
}  // namespace pat
