/*
 * pat_unet.h - C ABI of the learned warm start for the PDHG reconstruction of pat.h.
 *
 * The paper starts Algorithms 1 and 2 from zero iterates.  The learned warm start predicts
 * the converged iterates (u, v, r, s) of a reconstruction from its data with a U-Net
 * (Ronneberger, Fischer and Brox 2015).  q follows from the optimality condition of the
 * data term: q = K u - f, the fixed point of the prox of Sec. 3.2.  PDHG then runs from
 * that state to the same duality-gap tolerance (Sec. 3.3.3) as a cold start.  The network
 * is trained on the GPU by the kernels behind this header, on pairs that the PDHG solver
 * of pat.h generates.
 *
 * Network (all convolutions 3x3, zero padding, stride 1):
 *  - L levels with C0 * 2^l channels at level l.
 *  - Encoder level l: conv + ReLU, conv + ReLU.  Level 0 reads the input; level l > 0
 *    reads the 2x2 mean pooling of level l-1's output.
 *  - Decoder level l = L-2 ... 0: conv + ReLU, conv + ReLU on the channel concatenation
 *    [nearest 2x upsampling of level l+1's output, encoder output of level l].
 *  - Head: one conv to the output channels, without ReLU.
 *
 * Numerics:
 *  - Weights and activations are stored as bfloat16, and every sum accumulates in FP32
 *    on the tensor cores.
 *  - Biases, the head output, weight gradients, the FP32 master weights and the Adam
 *    moments are FP32.
 *
 * Layouts:
 *  - Activations are channels-last (NHWC): x[((n*H + iy)*W + ix)*C + c].
 *  - Weights are [c_out][ky][kx][c_in], applied as a cross-correlation:
 *    y[n,iy,ix,o] = b[o] + sum w[o,ky,kx,c] x[n, iy+ky-1, ix+kx-1, c].
 *  - bfloat16 values are passed as their 16-bit patterns (uint16_t).
 *  - The flat parameter vector lists the convolutions in the order enc0a, enc0b, ...,
 *    enc(L-1)b, dec(L-2)a, dec(L-2)b, ..., dec0b, head.  Each conv contributes its
 *    weights [c_out][3][3][c_in] followed by its bias [c_out].
 *
 * Conventions are those of pat.h:
 *  - *_dev pointers are caller-owned device memory;
 *  - calls are stream-ordered;
 *  - the return value is PAT_OK or a negative PAT_ERR_* code;
 *  - there is no CPU fallback.
 * A pat_unet must not be used by two calls at the same time.
 */
#ifndef PAT_UNET_H
#define PAT_UNET_H

#include <stdint.h>
#include "pat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- single convolutions (the network's building blocks; inputs bfloat16) -------- */

/* y = conv3x3(x, w) + bias, then max(y, 0) if relu != 0.  x: batch x h x w x cin (bf16),
   w: cout x 3 x 3 x cin (bf16), bias: cout FP32 or NULL, y: batch x h x w x cout FP32.
   cin and cout must be positive multiples of 8; x, w and y 16-byte aligned (checked). */
int pat_conv3x3_forward(const uint16_t* x_dev, int batch, int h, int w, int cin,
                        const uint16_t* w_dev, const float* bias_dev, int cout, int relu,
                        float* y_dev, void* stream);

/* dx = dL/dx of y = conv3x3(x, w) given dy = dL/dy (bf16, batch x h x w x cout):
   dx[n,iy,ix,c] = sum w[o,ky,kx,c] dy[n, iy-ky+1, ix-kx+1, o].  dx: FP32 NHWC, cin. */
int pat_conv3x3_backward_data(const uint16_t* dy_dev, int batch, int h, int w, int cout,
                              const uint16_t* w_dev, int cin, float* dx_dev, void* stream);

/* dw[o,ky,kx,c] = sum_{n,iy,ix} dy[n,iy,ix,o] x[n, iy+ky-1, ix+kx-1, c] and
   db[o] = sum dy[n,iy,ix,o] (FP32, overwritten; db may be NULL). */
int pat_conv3x3_backward_weight(const uint16_t* x_dev, const uint16_t* dy_dev, int batch, int h,
                                int w, int cin, int cout, float* dw_dev, float* db_dev,
                                void* stream);

/* Number of bounded waits in the tensor-memory convolutions (pat_conv3x3_forward,
   pat_conv3x3_backward_data and the network's forward and data-gradient passes) that ran
   out since the library was loaded.  Each such wait ends its CTA early: it counts here,
   drains its copies, frees its tensor memory and writes no output.  0 in normal operation.
   Returns PAT_OK, or PAT_ERR_CUDA if the counter cannot be read; count receives it. */
int pat_nn_wait_timeouts(unsigned* count);

/* ---- the network ------------------------------------------------------------------ */
typedef struct pat_unet pat_unet;   /* opaque */

typedef struct {
    int in_ch;                /* input channels, multiple of 8                          */
    int out_ch;               /* output channels, multiple of 8                         */
    int base_ch;              /* C0, channels at level 0, multiple of 8                 */
    int levels;               /* L >= 1; h and w of every call must be multiples of 2^(L-1) */
    unsigned long long seed;  /* initialisation: He-normal weights, std sqrt(2/(9 c_in)),
                                 from a SplitMix64 stream; zero biases                   */
} pat_unet_desc;

/* Creates the network on the current device.  Returns PAT_ERR_INVALID_ARG for channel
   counts that are not positive multiples of 8 or levels outside 1..8. */
int  pat_unet_create(const pat_unet_desc* desc, pat_unet** out);
void pat_unet_destroy(pat_unet* net);
long long pat_unet_num_params(const pat_unet* net);

/* Copy the FP32 master parameters (flat order above) to or from host memory.  Both
   synchronise the device.  set_params also resets the Adam moments and step count. */
int pat_unet_get_params(const pat_unet* net, float* params_host);
int pat_unet_set_params(pat_unet* net, const float* params_host);

/* y = net(x).  x: batch x h x w x in_ch (bf16), y: batch x h x w x out_ch (FP32).  The
   activations are kept inside the network for a following pat_unet_backward. */
int pat_unet_forward(pat_unet* net, const uint16_t* x_dev, int batch, int h, int w,
                     float* y_dev, void* stream);

/* Parameter gradient of the last forward call given dy = dL/dy (FP32, shape of y):
   grad_dev receives num_params FP32 values in the flat order.  dy is rounded to
   bfloat16 before it enters the backward convolutions. */
int pat_unet_backward(pat_unet* net, const float* dy_dev, float* grad_dev, void* stream);

/* One training step on a batch:
   - forward;
   - loss L = sum_c w_c sum (y - t)^2 / (batch h w out_ch), with ch_weight_host holding
     out_ch weights w_c;
   - backward;
   - one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with rate lr on
     the FP32 master parameters, then the bf16 copies are refreshed.
   loss_dev (1 FP32, may be NULL) receives L of this batch before the step. */
int pat_unet_train_step(pat_unet* net, const uint16_t* x_dev, const float* target_dev,
                        const float* ch_weight_host, int batch, int h, int w, float lr,
                        float* loss_dev, void* stream);

/* ---- the warm start ------------------------------------------------------------------ */
/* Normalisation of the 8 prediction channels (TGV; TV and dTV leave v and s zero):
   c0 = u, c1..2 = PAT_WARM_V_SCALE * v, c3..4 = r / alpha, c5..7 = s / (alpha beta). */
#define PAT_WARM_CHANNELS 8
#define PAT_WARM_V_SCALE  10.0f

/* Network input for data f (D*T FP32) on geometry g, written to x_dev (N x N x in_ch bf16,
   in_ch >= 2, a multiple of 8):
   - c0 = T K^T (S f) with T = 1/(K^T 1) per pixel and S = 1/(K 1) per data row.  These
     are the diagonal scalings of K alone (Sec. 3.3.2, alpha = 1), so c0 has the scale of
     u.  A zero sum gives 0.
   - c1 = (K^T 1) / max (K^T 1), the geometry's sensitivity.
   - c >= 2 are 0. */
int pat_warm_start_features(const pat_geometry* g, const float* f_dev, uint16_t* x_dev, int in_ch,
                            void* stream);

/* PDHG starting state from a prediction (N x N x out_ch FP32, out_ch >= 8, channels as
   above), in the x0 / y0 layouts of pat_params:
   - u = c0;
   - v = (c1, c2) / PAT_WARM_V_SCALE (TGV);
   - r = the projection of alpha (c3, c4) onto the alpha-ball;
   - s = the projection of alpha beta (c5, c6, c7) onto the alpha beta-ball (TGV);
   - q = K u - f.
   p supplies reg, alpha and beta. */
int pat_warm_start_state(const pat_geometry* g, const float* pred_dev, int out_ch,
                         const pat_params* p, const float* f_dev, float* x0_dev, float* y0_dev,
                         void* stream);

/* Training target from a PDHG state (x, y in the pat_params layouts): the inverse of the
   normalisation above, N x N x out_ch FP32 (channels >= 8 are 0). */
int pat_warm_start_target(const pat_geometry* g, const float* x_dev, const float* y_dev,
                          const pat_params* p, float* target_dev, int out_ch, void* stream);

/* Features, forward and state in one call (batch of one).  Scratch comes from the
   stream-ordered pool. */
int pat_warm_start(const pat_geometry* g, pat_unet* net, const float* f_dev, const pat_params* p,
                   float* x0_dev, float* y0_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PAT_UNET_H */
