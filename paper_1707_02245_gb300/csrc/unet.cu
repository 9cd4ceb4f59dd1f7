// The learned warm start: the U-Net (forward, backward, Adam) built on the tensor-core
// convolutions of conv.cu, and the maps between PDHG states and the network's channels.
//
// Dataflow of one training step (B images of H x W, L levels, C_l = C0 2^l channels):
//  - Forward:
//    - encoder l: [pool] -> conv a -> conv b.  The output of conv b is written straight
//      into the skip slice of the decoder's concatenation buffer at level l.
//    - decoder l: upsample into the concatenation buffer -> conv a -> conv b.
//    - head: conv to FP32.
//  - Loss: the weighted squared error gives the bf16 gradient of the head output and the
//    loss in one pass.
//  - Backward:
//    - for every conv: mask the output gradient by its ReLU, form the weight gradient,
//      then the input gradient by the transposed convolution (flipped weights).
//    - A map that feeds two consumers sums their gradients once, before its mask.  The
//      upsampling adjoint (2x2 sum) and the pooling adjoint (1/4 replicate, added to the
//      skip slice) are the resampling kernel.
//  - Adam on the flat FP32 master parameters, which also refreshes the bf16 copies.
#include <algorithm>
#include <cmath>
#include <vector>

#include "nn_internal.cuh"
#include "pat_internal.cuh"
#include "pat_unet.h"
#include "stencil.cuh"

using namespace pat;
using pat::nn::bf16;
using pat::nn::View;

namespace {

constexpr int EW_THREADS = 256;

// ---------------------------------------------------------------------------------------
// elementwise kernels (8 channels = one 16-byte vector per thread)
// ---------------------------------------------------------------------------------------
struct Vec8 {
    float v[8];
};
__device__ __forceinline__ Vec8 ld8(const bf16* p) {
    const uint4 r = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&r);
    Vec8 o;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        o.v[2 * i] = f.x;
        o.v[2 * i + 1] = f.y;
    }
    return o;
}
__device__ __forceinline__ void st8(bf16* p, const Vec8& a) {
    uint4 r;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(a.v[2 * i], a.v[2 * i + 1]);
    *reinterpret_cast<uint4*>(p) = r;
}

// out = scale * (mode 0: sum of the 2x2 input block; mode 1: the input pixel (y/2, x/2))
//       [+ add], rounded once to bf16.  Output size B x Ho x Wo, C channels.
struct ResampleArgs {
    const bf16* in;
    int in_ps;
    bf16* out;
    int out_ps;
    const bf16* add;
    int add_ps;
    int B, Ho, Wo, C, mode;
    float scale;
};

__global__ void k_resample(const ResampleArgs a) {
    const int cv = a.C / 8;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)a.B * a.Ho * a.Wo * cv;
    if (i >= n) return;
    const int c = (int)(i % cv) * 8;
    const long long p = i / cv;
    const int x = (int)(p % a.Wo), y = (int)((p / a.Wo) % a.Ho);
    const long long img = p / ((long long)a.Wo * a.Ho);
    Vec8 r;
    if (a.mode == 0) {
        const int Wi = a.Wo * 2, Hi = a.Ho * 2;
        const long long base = (img * Hi + 2 * y) * Wi + 2 * x;
        const Vec8 a0 = ld8(a.in + base * a.in_ps + c), a1 = ld8(a.in + (base + 1) * a.in_ps + c);
        const Vec8 a2 = ld8(a.in + (base + Wi) * a.in_ps + c), a3 = ld8(a.in + (base + Wi + 1) * a.in_ps + c);
#pragma unroll
        for (int k = 0; k < 8; ++k) r.v[k] = a.scale * ((a0.v[k] + a1.v[k]) + (a2.v[k] + a3.v[k]));
    } else {
        const int Wi = a.Wo / 2, Hi = a.Ho / 2;
        const long long q = (img * Hi + y / 2) * Wi + x / 2;
        const Vec8 a0 = ld8(a.in + q * a.in_ps + c);
#pragma unroll
        for (int k = 0; k < 8; ++k) r.v[k] = a.scale * a0.v[k];
    }
    if (a.add) {
        const Vec8 b = ld8(a.add + p * a.add_ps + c);
#pragma unroll
        for (int k = 0; k < 8; ++k) r.v[k] += b.v[k];
    }
    st8(a.out + p * a.out_ps + c, r);
}

// g <- g * [y > 0]  (the derivative of a ReLU, taken from its output)
__global__ void k_relu_mask(bf16* g, int g_ps, const bf16* y, int y_ps, long long P, int C) {
    const int cv = C / 8;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * cv) return;
    const int c = (int)(i % cv) * 8;
    const long long p = i / cv;
    Vec8 a = ld8(g + p * g_ps + c);
    const Vec8 m = ld8(y + p * y_ps + c);
#pragma unroll
    for (int k = 0; k < 8; ++k) a.v[k] = m.v[k] > 0.f ? a.v[k] : 0.f;
    st8(g + p * g_ps + c, a);
}

// dpred = 2 w_c (y - t) / count (bf16) and per-block partial sums of w_c (y - t)^2
constexpr int LOSS_BLOCKS = 256;
__global__ void __launch_bounds__(EW_THREADS) k_mse(const float* __restrict__ y, const float* __restrict__ t,
                                                    const float* __restrict__ w, int C, long long n,
                                                    bf16* __restrict__ dpred, double* __restrict__ part) {
    const double inv = 1.0 / (double)n;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const float d = y[i] - t[i];
        const float wd = w[c] * d;
        dpred[i] = __float2bfloat16_rn((float)(2.0 * inv) * wd);
        s += (double)(wd * d);
    }
    __shared__ double sh[EW_THREADS];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = EW_THREADS / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0] * inv;
}

__global__ void k_sum_partials(const double* __restrict__ part, int n, float* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = (float)s;
    }
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, bf16* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// Adam (Kingma and Ba 2015) with bias correction bc1 = 1 - beta1^t, bc2 = 1 - beta2^t;
// also writes the bf16 copy used by the convolutions.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, bf16* __restrict__ wb, long long n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

// ---------------------------------------------------------------------------------------
// warm-start maps
// ---------------------------------------------------------------------------------------
__global__ void k_div_or_zero(const float* __restrict__ num, const float* __restrict__ den, float* __restrict__ out,
                              long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = den[i] > 0.f ? num[i] / den[i] : 0.f;
}

__global__ void k_max_one_block(const float* __restrict__ x, long long n, float* __restrict__ out) {
    __shared__ float sh[EW_THREADS];
    float m = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, x[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int k = EW_THREADS / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// x[p][0] = T K^T S f, x[p][1] = K^T 1 / max, x[p][c >= 2] = 0
__global__ void k_features(const float* __restrict__ kt_sf, const float* __restrict__ kcol,
                           const float* __restrict__ kmax, bf16* __restrict__ x, long long NN, int in_ch) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NN) return;
    const float kc = kcol[p];
    const float mx = *kmax;
    for (int c0 = 0; c0 < in_ch; c0 += 8) {
        Vec8 v;
#pragma unroll
        for (int k = 0; k < 8; ++k) v.v[k] = 0.f;
        if (c0 == 0) {
            v.v[0] = kc > 0.f ? kt_sf[p] / kc : 0.f;
            v.v[1] = mx > 0.f ? kc / mx : 0.f;
        }
        st8(x + p * in_ch + c0, v);
    }
}

// prediction channels -> (u, v) and (r, s); q is formed afterwards as K u - f
__global__ void k_state(const float* __restrict__ pred, int C, long long NN, int reg, float alpha, float ab,
                        float* __restrict__ x0, float* __restrict__ rs) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NN) return;
    const float* c = pred + p * C;
    x0[p] = c[0];
    float r1 = alpha * c[3], r2 = alpha * c[4];
    proj2(r1, r2, alpha);
    rs[p] = r1;
    rs[NN + p] = r2;
    if (reg == PAT_TGV) {
        x0[NN + p] = c[1] / PAT_WARM_V_SCALE;
        x0[2 * NN + p] = c[2] / PAT_WARM_V_SCALE;
        float s11 = ab * c[5], s22 = ab * c[6], s12 = ab * c[7];
        proj3(s11, s22, s12, ab);
        rs[2 * NN + p] = s11;
        rs[3 * NN + p] = s22;
        rs[4 * NN + p] = s12;
    }
}

__global__ void k_sub_inplace(float* __restrict__ y, const float* __restrict__ f, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] -= f[i];
}

__global__ void k_target(const float* __restrict__ x, const float* __restrict__ rs, long long NN, int reg,
                         float inv_alpha, float inv_ab, float* __restrict__ t, int C) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NN) return;
    float* o = t + p * C;
    for (int c = 0; c < C; ++c) o[c] = 0.f;
    o[0] = x[p];
    o[3] = rs[p] * inv_alpha;
    o[4] = rs[NN + p] * inv_alpha;
    if (reg == PAT_TGV) {
        o[1] = x[NN + p] * PAT_WARM_V_SCALE;
        o[2] = x[2 * NN + p] * PAT_WARM_V_SCALE;
        o[5] = rs[2 * NN + p] * inv_ab;
        o[6] = rs[3 * NN + p] * inv_ab;
        o[7] = rs[4 * NN + p] * inv_ab;
    }
}

unsigned blocks_for(long long n) { return (unsigned)((n + EW_THREADS - 1) / EW_THREADS); }

#define NN_LAUNCH(kernel, n, st, ...)                                 \
    do {                                                             \
        kernel<<<blocks_for(n), EW_THREADS, 0, st>>>(__VA_ARGS__);   \
        PAT_LAUNCH_CHECK(#kernel);                                   \
    } while (0)

int resample(const View& in, const View& out, const View* add, int B, int Ho, int Wo, int C, int mode, float scale,
             cudaStream_t st) {
    ResampleArgs a;
    a.in = in.p;
    a.in_ps = in.ps;
    a.out = out.p;
    a.out_ps = out.ps;
    a.add = add ? add->p : nullptr;
    a.add_ps = add ? add->ps : 0;
    a.B = B;
    a.Ho = Ho;
    a.Wo = Wo;
    a.C = C;
    a.mode = mode;
    a.scale = scale;
    NN_LAUNCH(k_resample, (long long)B * Ho * Wo * (C / 8), st, a);
    return PAT_OK;
}

int relu_mask(const View& g, const View& y, long long P, int C, cudaStream_t st) {
    NN_LAUNCH(k_relu_mask, P * (C / 8), st, g.p, g.ps, y.p, y.ps, P, C);
    return PAT_OK;
}

// SplitMix64 (Steele, Lea and Flood 2014): a counter-based 64-bit generator.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() {   // Box-Muller
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

}  // namespace

// ---------------------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------------------
struct ConvSpec {
    int cout, cin;
    size_t w_off, b_off;   // offsets into the flat parameter vector
};

struct pat_unet {
    pat_unet_desc d;
    int device = 0;
    std::vector<ConvSpec> convs;
    long long nparams = 0;
    float* master = nullptr;   // FP32 parameters (flat)
    float* mom1 = nullptr;
    float* mom2 = nullptr;
    float* grad = nullptr;
    bf16* wbf = nullptr;       // bf16 copy (same offsets; bias slots unused)
    bf16* wflip = nullptr;     // flipped weights of one conv (largest size)
    float* chw = nullptr;      // loss channel weights (out_ch)
    long long step = 0;
    // activations and gradients for the current (B, H, W)
    int aB = 0, aH = 0, aW = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<bf16*> pin, A, cat, DA, D, gD, gDA, gcat, gE, gA, gIn;
    bf16* ebot = nullptr;
    bf16* gEbot = nullptr;
    bf16* dpred = nullptr;
    float* ypred = nullptr;
    float* wpart = nullptr;
    double* loss_part = nullptr;
    const bf16* x_last = nullptr;   // input of the last forward
    bool have_forward = false;
};

namespace {

int ch(const pat_unet* net, int l) { return net->d.base_ch << l; }
int cat_ch(const pat_unet* net, int l) { return ch(net, l + 1) + ch(net, l); }
int conv_enc(int l, int which) { return 2 * l + which; }
int conv_dec(const pat_unet* net, int l, int which) { return 2 * net->d.levels + 2 * (net->d.levels - 2 - l) + which; }
int conv_head(const pat_unet* net) { return 4 * net->d.levels - 2; }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int ensure_workspace(pat_unet* net, int B, int H, int W) {
    if (net->ws && net->aB == B && net->aH == H && net->aW == W) return PAT_OK;
    if (net->ws) {
        cudaFree(net->ws);
        net->ws = nullptr;
    }
    const int L = net->d.levels;
    std::vector<std::pair<void**, size_t>> req;
    auto add = [&](void** p, size_t bytes) { req.push_back({p, align256(bytes)}); };
    auto px = [&](int l) { return (size_t)B * (H >> l) * (W >> l); };
    net->pin.assign(L, nullptr);
    net->A.assign(L, nullptr);
    net->cat.assign(L, nullptr);
    net->DA.assign(L, nullptr);
    net->D.assign(L, nullptr);
    net->gD.assign(L, nullptr);
    net->gDA.assign(L, nullptr);
    net->gcat.assign(L, nullptr);
    net->gE.assign(L, nullptr);
    net->gA.assign(L, nullptr);
    net->gIn.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        const size_t P = px(l), Cl = ch(net, l);
        if (l > 0) {
            add((void**)&net->pin[l], P * ch(net, l - 1) * 2);
            add((void**)&net->gIn[l], P * ch(net, l - 1) * 2);
        }
        add((void**)&net->A[l], P * Cl * 2);
        add((void**)&net->gA[l], P * Cl * 2);
        if (l <= L - 2) {
            add((void**)&net->cat[l], P * cat_ch(net, l) * 2);
            add((void**)&net->gcat[l], P * cat_ch(net, l) * 2);
            add((void**)&net->DA[l], P * Cl * 2);
            add((void**)&net->D[l], P * Cl * 2);
            add((void**)&net->gD[l], P * Cl * 2);
            add((void**)&net->gDA[l], P * Cl * 2);
            add((void**)&net->gE[l], P * Cl * 2);
        }
    }
    add((void**)&net->ebot, px(L - 1) * ch(net, L - 1) * 2);
    add((void**)&net->gEbot, px(L - 1) * ch(net, L - 1) * 2);
    add((void**)&net->dpred, px(0) * net->d.out_ch * 2);
    add((void**)&net->ypred, px(0) * net->d.out_ch * 4);
    add((void**)&net->loss_part, LOSS_BLOCKS * 8 + 8);
    size_t wp = 0;
    for (int l = 0; l < L; ++l)
        for (const ConvSpec& c : net->convs) wp = std::max(wp, nn::wgrad_partial_floats(B, H >> l, W >> l, c.cin, c.cout));
    add((void**)&net->wpart, wp * 4);
    size_t total = 0;
    for (auto& r : req) total += r.second;
    char* base = nullptr;
    if (cudaMalloc(&base, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(PAT_ERR_OOM, "pat_unet: cannot allocate the activation workspace");
    }
    size_t off = 0;
    for (auto& r : req) {
        *r.first = base + off;
        off += r.second;
    }
    net->ws = base;
    net->ws_bytes = total;
    net->aB = B;
    net->aH = H;
    net->aW = W;
    net->have_forward = false;
    return PAT_OK;
}

View e_view(pat_unet* net, int l) {
    const int L = net->d.levels;
    if (l == L - 1) return View{net->ebot, ch(net, l)};
    return View{net->cat[l] + ch(net, l + 1), cat_ch(net, l)};
}
View level_out(pat_unet* net, int l) {   // output of level l as seen by the level above
    return l == net->d.levels - 1 ? e_view(net, l) : View{net->D[l], ch(net, l)};
}
View top_view(pat_unet* net) { return net->d.levels >= 2 ? View{net->D[0], ch(net, 0)} : e_view(net, 0); }

int conv(pat_unet* net, int idx, const View& x, int l, const View& y, bool relu, float* y32, cudaStream_t st) {
    const ConvSpec& c = net->convs[idx];
    return nn::conv3x3_fwd(x, net->aB, net->aH >> l, net->aW >> l, c.cin, net->wbf + c.w_off, net->master + c.b_off,
                           c.cout, relu, y, y32, c.cout, st);
}

// weight gradient into grad, and (if dx.p) the input gradient
int conv_back(pat_unet* net, int idx, const View& x, const View& dz, int l, const View& dx, float* grad,
              cudaStream_t st) {
    const ConvSpec& c = net->convs[idx];
    const int Hl = net->aH >> l, Wl = net->aW >> l;
    int rc = nn::conv3x3_wgrad(x, dz, net->aB, Hl, Wl, c.cin, c.cout, grad + c.w_off, grad + c.b_off, net->wpart, st);
    if (rc || !dx.p) return rc;
    rc = nn::flip_weights(net->wbf + c.w_off, c.cout, c.cin, net->wflip, st);
    if (rc) return rc;
    return nn::conv3x3_fwd(dz, net->aB, Hl, Wl, c.cout, net->wflip, nullptr, c.cin, false, dx, nullptr, 0, st);
}

#define TRY(x)                  \
    do {                        \
        int rc_ = (x);          \
        if (rc_) return rc_;    \
    } while (0)

int forward_impl(pat_unet* net, const bf16* x, int B, int H, int W, float* y, cudaStream_t st) {
    const int L = net->d.levels;
    TRY(ensure_workspace(net, B, H, W));
    View in{const_cast<bf16*>(x), net->d.in_ch};
    for (int l = 0; l < L; ++l) {
        if (l > 0) {
            const View pin{net->pin[l], ch(net, l - 1)};
            TRY(resample(e_view(net, l - 1), pin, nullptr, B, H >> l, W >> l, ch(net, l - 1), 0, 0.25f, st));
            in = pin;
        }
        const View a{net->A[l], ch(net, l)};
        TRY(conv(net, conv_enc(l, 0), in, l, a, true, nullptr, st));
        TRY(conv(net, conv_enc(l, 1), a, l, e_view(net, l), true, nullptr, st));
    }
    for (int l = L - 2; l >= 0; --l) {
        const View cat{net->cat[l], cat_ch(net, l)};
        TRY(resample(level_out(net, l + 1), cat, nullptr, B, H >> l, W >> l, ch(net, l + 1), 1, 1.f, st));
        const View da{net->DA[l], ch(net, l)};
        TRY(conv(net, conv_dec(net, l, 0), cat, l, da, true, nullptr, st));
        TRY(conv(net, conv_dec(net, l, 1), da, l, View{net->D[l], ch(net, l)}, true, nullptr, st));
    }
    TRY(conv(net, conv_head(net), top_view(net), 0, View{nullptr, 0}, false, y, st));
    net->x_last = x;
    net->have_forward = true;
    return PAT_OK;
}

int backward_impl(pat_unet* net, float* grad, cudaStream_t st) {
    const int L = net->d.levels;
    const int B = net->aB, H = net->aH, W = net->aW;
    auto P = [&](int l) { return (long long)B * (H >> l) * (W >> l); };
    const View g_top = L >= 2 ? View{net->gD[0], ch(net, 0)} : View{net->gEbot, ch(net, 0)};
    TRY(conv_back(net, conv_head(net), top_view(net), View{net->dpred, net->d.out_ch}, 0, g_top, grad, st));
    for (int l = 0; l <= L - 2; ++l) {
        const View gd{net->gD[l], ch(net, l)}, gda{net->gDA[l], ch(net, l)};
        const View da{net->DA[l], ch(net, l)}, d{net->D[l], ch(net, l)};
        const View cat{net->cat[l], cat_ch(net, l)}, gcat{net->gcat[l], cat_ch(net, l)};
        TRY(relu_mask(gd, d, P(l), ch(net, l), st));
        TRY(conv_back(net, conv_dec(net, l, 1), da, gd, l, gda, grad, st));
        TRY(relu_mask(gda, da, P(l), ch(net, l), st));
        TRY(conv_back(net, conv_dec(net, l, 0), cat, gda, l, gcat, grad, st));
        const View gnext = l + 1 <= L - 2 ? View{net->gD[l + 1], ch(net, l + 1)} : View{net->gEbot, ch(net, l + 1)};
        TRY(resample(gcat, gnext, nullptr, B, H >> (l + 1), W >> (l + 1), ch(net, l + 1), 0, 1.f, st));
    }
    for (int l = L - 1; l >= 0; --l) {
        View ge{net->gEbot, ch(net, l)};
        if (l < L - 1) {
            ge = View{net->gE[l], ch(net, l)};
            const View skip{net->gcat[l] + ch(net, l + 1), cat_ch(net, l)};
            TRY(resample(View{net->gIn[l + 1], ch(net, l)}, ge, &skip, B, H >> l, W >> l, ch(net, l), 1, 0.25f, st));
        }
        TRY(relu_mask(ge, e_view(net, l), P(l), ch(net, l), st));
        const View a{net->A[l], ch(net, l)}, ga{net->gA[l], ch(net, l)};
        TRY(conv_back(net, conv_enc(l, 1), a, ge, l, ga, grad, st));
        TRY(relu_mask(ga, a, P(l), ch(net, l), st));
        const View in = l > 0 ? View{net->pin[l], ch(net, l - 1)} : View{const_cast<bf16*>(net->x_last), net->d.in_ch};
        const View gin = l > 0 ? View{net->gIn[l], ch(net, l - 1)} : View{nullptr, 0};
        TRY(conv_back(net, conv_enc(l, 0), in, ga, l, gin, grad, st));
    }
    return PAT_OK;
}

int check_shape(const pat_unet* net, int B, int H, int W) {
    const int m = 1 << (net->d.levels - 1);
    if (B <= 0 || H <= 0 || W <= 0 || H % m || W % m)
        return fail(PAT_ERR_INVALID_ARG, "pat_unet: batch, h, w must be positive and h, w multiples of 2^(levels-1)");
    return PAT_OK;
}

int set_device(const pat_unet* net) {
    PAT_CUDA(cudaSetDevice(net->device));
    return PAT_OK;
}

bool mult8(int c) { return c > 0 && c % 8 == 0; }
bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

int pat_nn_wait_timeouts(unsigned* count) {
    if (!count) return fail(PAT_ERR_INVALID_ARG, "pat_nn_wait_timeouts: null argument");
    *count = nn::wait_timeouts();
    return *count == ~0u ? fail(PAT_ERR_CUDA, "pat_nn_wait_timeouts: counter not readable") : PAT_OK;
}

int pat_conv3x3_forward(const uint16_t* x_dev, int batch, int h, int w, int cin, const uint16_t* w_dev,
                        const float* bias_dev, int cout, int relu, float* y_dev, void* stream) {
    if (!x_dev || !w_dev || !y_dev || batch < 0 || h < 0 || w < 0 || !mult8(cin) || !mult8(cout))
        return fail(PAT_ERR_INVALID_ARG, "pat_conv3x3_forward: null pointer, negative size or channels not a multiple of 8");
    if (!aligned16(x_dev) || !aligned16(w_dev) || !aligned16(y_dev))
        return fail(PAT_ERR_INVALID_ARG, "pat_conv3x3_forward: x, w and y must be 16-byte aligned");
    const View x{(bf16*)x_dev, cin};
    return nn::conv3x3_fwd(x, batch, h, w, cin, (const bf16*)w_dev, bias_dev, cout, relu != 0, View{nullptr, 0}, y_dev,
                           cout, (cudaStream_t)stream);
}

int pat_conv3x3_backward_data(const uint16_t* dy_dev, int batch, int h, int w, int cout, const uint16_t* w_dev, int cin,
                              float* dx_dev, void* stream) {
    if (!dy_dev || !w_dev || !dx_dev || batch < 0 || h < 0 || w < 0 || !mult8(cin) || !mult8(cout) ||
        !aligned16(dy_dev) || !aligned16(w_dev) || !aligned16(dx_dev))
        return fail(PAT_ERR_INVALID_ARG, "pat_conv3x3_backward_data: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    bf16* wf = nullptr;
    PAT_CUDA(cudaMallocAsync(&wf, (size_t)cout * 9 * cin * 2, st));
    int rc = nn::flip_weights((const bf16*)w_dev, cout, cin, wf, st);
    if (!rc)
        rc = nn::conv3x3_fwd(View{(bf16*)dy_dev, cout}, batch, h, w, cout, wf, nullptr, cin, false, View{nullptr, 0},
                             dx_dev, cin, st);
    cudaFreeAsync(wf, st);
    return rc;
}

int pat_conv3x3_backward_weight(const uint16_t* x_dev, const uint16_t* dy_dev, int batch, int h, int w, int cin,
                                int cout, float* dw_dev, float* db_dev, void* stream) {
    if (!x_dev || !dy_dev || !dw_dev || batch < 0 || h < 0 || w < 0 || !mult8(cin) || !mult8(cout))
        return fail(PAT_ERR_INVALID_ARG, "pat_conv3x3_backward_weight: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    float* part = nullptr;
    PAT_CUDA(cudaMallocAsync(&part, nn::wgrad_partial_floats(batch, h, w, cin, cout) * 4 + 16, st));
    const int rc = nn::conv3x3_wgrad(View{(bf16*)x_dev, cin}, View{(bf16*)dy_dev, cout}, batch, h, w, cin, cout, dw_dev,
                                     db_dev, part, st);
    cudaFreeAsync(part, st);
    return rc;
}

int pat_unet_create(const pat_unet_desc* desc, pat_unet** out) {
    if (!desc || !out) return fail(PAT_ERR_INVALID_ARG, "pat_unet_create: null argument");
    *out = nullptr;
    if (!mult8(desc->in_ch) || !mult8(desc->out_ch) || !mult8(desc->base_ch) || desc->levels < 1 || desc->levels > 8)
        return fail(PAT_ERR_INVALID_ARG,
                    "pat_unet_create: channel counts must be positive multiples of 8 and levels in 1..8");
    pat_unet* net = new pat_unet();
    net->d = *desc;
    PAT_CUDA(cudaGetDevice(&net->device));
    const int L = desc->levels;
    auto addc = [&](int cout, int cin) {
        ConvSpec c;
        c.cout = cout;
        c.cin = cin;
        c.w_off = (size_t)net->nparams;
        c.b_off = c.w_off + (size_t)cout * 9 * cin;
        net->nparams = (long long)(c.b_off + cout);
        net->convs.push_back(c);
    };
    int cin = desc->in_ch;
    for (int l = 0; l < L; ++l) {
        addc(ch(net, l), cin);
        addc(ch(net, l), ch(net, l));
        cin = ch(net, l);
    }
    for (int l = L - 2; l >= 0; --l) {
        addc(ch(net, l), cat_ch(net, l));
        addc(ch(net, l), ch(net, l));
    }
    addc(desc->out_ch, ch(net, 0));
    // He-normal initialisation from the seed, zero biases
    std::vector<float> h((size_t)net->nparams, 0.f);
    SplitMix64 rng{desc->seed};
    size_t maxw = 0;
    for (const ConvSpec& c : net->convs) {
        const double sd = std::sqrt(2.0 / (9.0 * c.cin));
        const size_t nw = (size_t)c.cout * 9 * c.cin;
        for (size_t i = 0; i < nw; ++i) h[c.w_off + i] = (float)(sd * rng.normal());
        maxw = std::max(maxw, nw);
    }
    const size_t n = (size_t)net->nparams;
    bool ok = cudaMalloc(&net->master, n * 4) == cudaSuccess && cudaMalloc(&net->mom1, n * 4) == cudaSuccess &&
              cudaMalloc(&net->mom2, n * 4) == cudaSuccess && cudaMalloc(&net->grad, n * 4) == cudaSuccess &&
              cudaMalloc(&net->wbf, n * 2) == cudaSuccess && cudaMalloc(&net->wflip, maxw * 2) == cudaSuccess &&
              cudaMalloc(&net->chw, (size_t)desc->out_ch * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pat_unet_destroy(net);
        return fail(PAT_ERR_OOM, "pat_unet_create: out of device memory");
    }
    *out = net;
    const int rc = pat_unet_set_params(net, h.data());
    if (rc) {
        pat_unet_destroy(net);
        *out = nullptr;
    }
    return rc;
}

void pat_unet_destroy(pat_unet* net) {
    if (!net) return;
    cudaSetDevice(net->device);
    cudaFree(net->master);
    cudaFree(net->mom1);
    cudaFree(net->mom2);
    cudaFree(net->grad);
    cudaFree(net->wbf);
    cudaFree(net->wflip);
    cudaFree(net->chw);
    cudaFree(net->ws);
    delete net;
}

long long pat_unet_num_params(const pat_unet* net) { return net ? net->nparams : -1; }

int pat_unet_get_params(const pat_unet* net, float* params_host) {
    if (!net || !params_host) return fail(PAT_ERR_INVALID_ARG, "pat_unet_get_params: null argument");
    TRY(set_device(net));
    PAT_CUDA(cudaDeviceSynchronize());
    PAT_CUDA(cudaMemcpy(params_host, net->master, (size_t)net->nparams * 4, cudaMemcpyDeviceToHost));
    return PAT_OK;
}

int pat_unet_set_params(pat_unet* net, const float* params_host) {
    if (!net || !params_host) return fail(PAT_ERR_INVALID_ARG, "pat_unet_set_params: null argument");
    TRY(set_device(net));
    const size_t n = (size_t)net->nparams;
    PAT_CUDA(cudaDeviceSynchronize());
    PAT_CUDA(cudaMemcpy(net->master, params_host, n * 4, cudaMemcpyHostToDevice));
    PAT_CUDA(cudaMemset(net->mom1, 0, n * 4));
    PAT_CUDA(cudaMemset(net->mom2, 0, n * 4));
    k_f32_to_bf16<<<blocks_for((long long)n), EW_THREADS>>>(net->master, net->wbf, (long long)n);
    PAT_LAUNCH_CHECK("k_f32_to_bf16");
    PAT_CUDA(cudaDeviceSynchronize());
    net->step = 0;
    return PAT_OK;
}

int pat_unet_forward(pat_unet* net, const uint16_t* x_dev, int batch, int h, int w, float* y_dev, void* stream) {
    if (!net || !x_dev || !y_dev) return fail(PAT_ERR_INVALID_ARG, "pat_unet_forward: null argument");
    TRY(check_shape(net, batch, h, w));
    return forward_impl(net, (const bf16*)x_dev, batch, h, w, y_dev, (cudaStream_t)stream);
}

int pat_unet_backward(pat_unet* net, const float* dy_dev, float* grad_dev, void* stream) {
    if (!net || !dy_dev || !grad_dev) return fail(PAT_ERR_INVALID_ARG, "pat_unet_backward: null argument");
    if (!net->have_forward) return fail(PAT_ERR_INVALID_ARG, "pat_unet_backward: no forward call to differentiate");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)net->aB * net->aH * net->aW * net->d.out_ch;
    NN_LAUNCH(k_f32_to_bf16, n, st, dy_dev, net->dpred, n);
    return backward_impl(net, grad_dev, st);
}

int pat_unet_train_step(pat_unet* net, const uint16_t* x_dev, const float* target_dev, const float* ch_weight_host,
                        int batch, int h, int w, float lr, float* loss_dev, void* stream) {
    if (!net || !x_dev || !target_dev || !ch_weight_host)
        return fail(PAT_ERR_INVALID_ARG, "pat_unet_train_step: null argument");
    TRY(check_shape(net, batch, h, w));
    cudaStream_t st = (cudaStream_t)stream;
    PAT_CUDA(cudaMemcpyAsync(net->chw, ch_weight_host, (size_t)net->d.out_ch * 4, cudaMemcpyHostToDevice, st));
    TRY(ensure_workspace(net, batch, h, w));
    TRY(forward_impl(net, (const bf16*)x_dev, batch, h, w, net->ypred, st));
    const long long n = (long long)batch * h * w * net->d.out_ch;
    k_mse<<<LOSS_BLOCKS, EW_THREADS, 0, st>>>(net->ypred, target_dev, net->chw, net->d.out_ch, n, net->dpred,
                                              net->loss_part);
    PAT_LAUNCH_CHECK("k_mse");
    if (loss_dev) {
        k_sum_partials<<<1, 32, 0, st>>>(net->loss_part, LOSS_BLOCKS, loss_dev);
        PAT_LAUNCH_CHECK("k_sum_partials");
    }
    TRY(backward_impl(net, net->grad, st));
    net->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 - std::pow(b1, (double)net->step));
    const float bc2 = (float)(1.0 - std::pow(b2, (double)net->step));
    NN_LAUNCH(k_adam, net->nparams, st, net->master, net->mom1, net->mom2, net->grad, net->wbf, net->nparams, lr,
              (float)b1, (float)b2, 1e-8f, bc1, bc2);
    return PAT_OK;
}

int pat_warm_start_features(const pat_geometry* g, const float* f_dev, uint16_t* x_dev, int in_ch, void* stream) {
    if (!g || !f_dev || !x_dev || !mult8(in_ch))
        return fail(PAT_ERR_INVALID_ARG, "pat_warm_start_features: null argument or in_ch not a positive multiple of 8");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(ensure_precond(g, st));
    const long long NN = (long long)g->desc.n * g->desc.n;
    const long long S = (long long)g->desc.n_det * g->desc.n_t;
    float* scratch = nullptr;
    PAT_CUDA(cudaMallocAsync(&scratch, (size_t)(S + NN + 64) * 4, st));
    float* sf = scratch;
    float* kt = scratch + S;
    float* kmax = scratch + S + NN;
    int rc = PAT_OK;
    k_div_or_zero<<<blocks_for(S), EW_THREADS, 0, st>>>(f_dev, g->pc.krow, sf, S);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = fail(PAT_ERR_CUDA, "k_div_or_zero launch failed");
    if (!rc) rc = launch_adjoint(g, sf, kt, st);
    if (!rc) {
        k_max_one_block<<<1, EW_THREADS, 0, st>>>(g->pc.kcol, NN, kmax);
        k_features<<<blocks_for(NN), EW_THREADS, 0, st>>>(kt, g->pc.kcol, kmax, (bf16*)x_dev, NN, in_ch);
        count_launch();
        count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = fail(PAT_ERR_CUDA, "k_features launch failed");
    }
    cudaFreeAsync(scratch, st);
    return rc;
}

int pat_warm_start_state(const pat_geometry* g, const float* pred_dev, int out_ch, const pat_params* p,
                         const float* f_dev, float* x0_dev, float* y0_dev, void* stream) {
    if (!g || !pred_dev || !p || !f_dev || !x0_dev || !y0_dev || out_ch < PAT_WARM_CHANNELS)
        return fail(PAT_ERR_INVALID_ARG, "pat_warm_start_state: null argument or out_ch < 8");
    if (p->reg < PAT_TV || p->reg > PAT_DTV || !(p->alpha > 0.0) || (p->reg == PAT_TGV && !(p->beta > 0.0)))
        return fail(PAT_ERR_INVALID_ARG, "pat_warm_start_state: invalid regulariser or parameters");
    cudaStream_t st = (cudaStream_t)stream;
    const long long NN = (long long)g->desc.n * g->desc.n;
    const long long S = (long long)g->desc.n_det * g->desc.n_t;
    NN_LAUNCH(k_state, NN, st, pred_dev, out_ch, NN, p->reg, (float)p->alpha, (float)(p->alpha * p->beta), x0_dev,
              y0_dev + S);
    TRY(launch_forward(g, x0_dev, y0_dev, st));
    NN_LAUNCH(k_sub_inplace, S, st, y0_dev, f_dev, S);
    return PAT_OK;
}

int pat_warm_start_target(const pat_geometry* g, const float* x_dev, const float* y_dev, const pat_params* p,
                          float* target_dev, int out_ch, void* stream) {
    if (!g || !x_dev || !y_dev || !p || !target_dev || out_ch < PAT_WARM_CHANNELS)
        return fail(PAT_ERR_INVALID_ARG, "pat_warm_start_target: null argument or out_ch < 8");
    if (p->reg < PAT_TV || p->reg > PAT_DTV || !(p->alpha > 0.0) || (p->reg == PAT_TGV && !(p->beta > 0.0)))
        return fail(PAT_ERR_INVALID_ARG, "pat_warm_start_target: invalid regulariser or parameters");
    cudaStream_t st = (cudaStream_t)stream;
    const long long NN = (long long)g->desc.n * g->desc.n;
    const long long S = (long long)g->desc.n_det * g->desc.n_t;
    const double ab = p->reg == PAT_TGV ? p->alpha * p->beta : 1.0;
    NN_LAUNCH(k_target, NN, st, x_dev, y_dev + S, NN, p->reg, (float)(1.0 / p->alpha), (float)(1.0 / ab), target_dev,
              out_ch);
    return PAT_OK;
}

int pat_warm_start(const pat_geometry* g, pat_unet* net, const float* f_dev, const pat_params* p, float* x0_dev,
                   float* y0_dev, void* stream) {
    if (!g || !net || !f_dev || !p || !x0_dev || !y0_dev) return fail(PAT_ERR_INVALID_ARG, "pat_warm_start: null argument");
    const int N = g->desc.n;
    TRY(check_shape(net, 1, N, N));
    if (net->d.out_ch < PAT_WARM_CHANNELS || net->d.in_ch < 8)
        return fail(PAT_ERR_INVALID_ARG, "pat_warm_start: the network needs >= 8 output channels");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t NN = (size_t)N * N;
    char* scratch = nullptr;
    const size_t xb = align256(NN * net->d.in_ch * 2);
    PAT_CUDA(cudaMallocAsync(&scratch, xb + NN * net->d.out_ch * 4, st));
    bf16* x = (bf16*)scratch;
    float* pred = (float*)(scratch + xb);
    int rc = pat_warm_start_features(g, f_dev, (uint16_t*)x, net->d.in_ch, stream);
    if (!rc) rc = forward_impl(net, x, 1, N, N, pred, st);
    if (!rc) rc = pat_warm_start_state(g, pred, net->d.out_ch, p, f_dev, x0_dev, y0_dev, stream);
    net->have_forward = false;   // the input buffer is released below
    cudaFreeAsync(scratch, st);
    return rc;
}

}  // extern "C"
