// Measurement pre-processing of Sec. 4.3: per detector, the regularised deconvolution of
// the pressure by the calibration measurement moved to the retarded time (eq. (deconv),
// eq. (FW_full)), then the rescale f = t / |x_d - x_p| f_t (eq. (f_rewrite)).
//
// One CTA per detector.  Both signals are zero-padded to L = the smallest power of two
// >= 2T (so that the spectral product stands for a linear convolution) and transformed by
// an in-shared-memory radix-2 FFT (iterative Cooley-Tukey, bit-reversed load).  The
// calibration is advanced by its travel time with the shift theorem: its spectrum is
// multiplied by exp(+2 pi i nu delta / L), with nu the signed frequency and delta the
// delay in samples; at the Nyquist index only the cosine is kept.  The regularisation is
// eps = eps_rel * max |F{dr h}|^2 of the detector.
#include <cmath>
#include <vector>

#include "pat_internal.cuh"

namespace pat {
namespace {

constexpr int PREP_THREADS = 512;
constexpr int PREP_MAX_L = 4096;   // T <= 2048

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// In-place radix-2 FFT of length L (a power of two) in shared memory; the data must have
// been stored in bit-reversed order.  sign = -1: forward, +1: inverse (unnormalised).
__device__ void fft_shared(float2* a, int L, int logL, float sign) {
    for (int s = 1; s <= logL; ++s) {
        const int m = 1 << s, half = m >> 1;
        for (int b = threadIdx.x; b < L / 2; b += blockDim.x) {
            const int grp = b / half, j = b - grp * half;
            const int i0 = grp * m + j, i1 = i0 + half;
            float sn, cs;
            sincospif(sign * 2.0f * (float)j / (float)m, &sn, &cs);
            const float2 t = cmul(make_float2(cs, sn), a[i1]);
            const float2 u = a[i0];
            a[i0] = make_float2(u.x + t.x, u.y + t.y);
            a[i1] = make_float2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

struct PrepArgs {
    const float* p;       // D x T
    const float* pcal;    // D x T
    const double* dist;   // D: |x_d - x_p|
    float* f;             // D x T
    int T, L, logL;
    double r0, dr, eps_rel;
};

__global__ void __launch_bounds__(PREP_THREADS) k_preprocess(const PrepArgs a) {
    extern __shared__ float2 sh[];
    float2* A = sh;           // pressure
    float2* B = sh + a.L;     // calibration
    __shared__ float s_max[PREP_THREADS / 32];
    const int d = blockIdx.x, T = a.T, L = a.L;
    const float* pd = a.p + (size_t)d * T;
    const float* cd = a.pcal + (size_t)d * T;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int r = (int)(__brev((unsigned)i) >> (32 - a.logL));   // bit-reversed position
        A[r] = make_float2(i < T ? pd[i] : 0.f, 0.f);
        B[r] = make_float2(i < T ? cd[i] : 0.f, 0.f);
    }
    __syncthreads();
    fft_shared(A, L, a.logL, -1.f);
    fft_shared(B, L, a.logL, -1.f);
    // H = dr * F{p_cal} * exp(+2 pi i nu delta / L), delta = (dist - t0) / dr
    const double t0 = a.r0 + 0.5 * a.dr;
    const double delta = (a.dist[d] - t0) / a.dr;
    float mx = 0.f;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int nu = i < L / 2 ? i : i - L;
        // the phase's argument reduced in FP64 (delta * nu can be large), then one FP32 sincos
        const double turns = (double)nu * delta / (double)L;
        const float fr = (float)(2.0 * (turns - rint(turns)));
        float sn, cs;
        sincospif(fr, &sn, &cs);
        if (i == L / 2) {
            sn = 0.f;
            cs = cospif((float)(delta - 2.0 * rint(0.5 * delta)));
        }
        const float2 h = cmul(B[i], make_float2(cs, sn));
        const float2 hd = make_float2((float)a.dr * h.x, (float)a.dr * h.y);
        B[i] = hd;
        mx = fmaxf(mx, hd.x * hd.x + hd.y * hd.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? s_max[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) s_max[0] = v;
    }
    __syncthreads();
    const float eps = (float)a.eps_rel * s_max[0];
    // F = P conj(H) / (|H|^2 + eps) in place in A, then into B in bit-reversed order for
    // the inverse transform
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const float2 h = B[i], pp = A[i];
        const float den = h.x * h.x + h.y * h.y + eps;
        A[i] = den > 0.f ? make_float2((pp.x * h.x + pp.y * h.y) / den, (pp.y * h.x - pp.x * h.y) / den)
                         : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += blockDim.x) B[(int)(__brev((unsigned)i) >> (32 - a.logL))] = A[i];
    __syncthreads();
    fft_shared(B, L, a.logL, 1.f);
    const double dist = a.dist[d];
    float* fd = a.f + (size_t)d * T;
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        const double t = a.r0 + (k + 0.5) * a.dr;
        fd[k] = (float)(t / dist * (double)B[k].x / (double)L);
    }
}

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" int pat_preprocess(const pat_geometry* g, const float* p_dev, const float* pcal_dev, const double* xp_host,
                              double eps_rel, float* f_dev, void* stream) {
    if (!g || !p_dev || !pcal_dev || !xp_host || !f_dev)
        return fail(PAT_ERR_INVALID_ARG, "pat_preprocess: NULL argument");
    if (!(eps_rel > 0) || !std::isfinite(eps_rel))
        return fail(PAT_ERR_INVALID_ARG, "pat_preprocess: eps_rel must be finite and > 0");
    const int D = g->desc.n_det, T = g->desc.n_t;
    if (T > PREP_MAX_L / 2) return fail(PAT_ERR_INVALID_ARG, "pat_preprocess: at most 2048 time samples");
    int L = 1, logL = 0;
    while (L < 2 * T) {
        L *= 2;
        ++logL;
    }
    std::vector<double> dist(D);
    for (int d = 0; d < D; ++d) {
        dist[d] = std::hypot(g->det_xy[2 * d] - xp_host[0], g->det_xy[2 * d + 1] - xp_host[1]);
        if (!(dist[d] > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_preprocess: the pulse source sits on a detector");
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* ddist = nullptr;
    PAT_CUDA(cudaMallocAsync(&ddist, D * sizeof(double), st));
    int rc = cudaMemcpyAsync(ddist, dist.data(), D * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess
                 ? PAT_OK
                 : fail(PAT_ERR_CUDA, "pat_preprocess: copy failed");
    if (!rc) {
        PrepArgs a{p_dev, pcal_dev, ddist, f_dev, T, L, logL, g->desc.r0, g->desc.dr, eps_rel};
        const size_t smem = 2 * (size_t)L * sizeof(float2);
        if (cudaFuncSetAttribute(k_preprocess, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            rc = fail(PAT_ERR_CUDA, "pat_preprocess: shared memory attribute");
        if (!rc) {
            k_preprocess<<<D, PREP_THREADS, smem, st>>>(a);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = fail(PAT_ERR_CUDA, "pat_preprocess: launch failed");
        }
    }
    cudaFreeAsync(ddist, st);
    return rc;
}
