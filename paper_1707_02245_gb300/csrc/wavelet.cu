// The wavelet model of Sec. 2.2 (eq. (min_wav)): W, its transpose, the |W| sums of the
// diagonal steps, and the pointwise kernels of the wavelet PDHG (Algorithm 1 with grad -> W
// and div -> -W^T, Sec. 3.3).
//
// W is the orthonormal separable 2-D Daubechies-4 transform with periodic extension and
// J levels in the Mallat layout: level l splits the top-left M x M block (M = N / 2^l)
// into LL (top-left), HL (top-right, high-pass along x), LH (bottom-left, high-pass
// along y) and HH.  It stands in for the paper's dual-tree complex wavelet transform (whose
// Q-shift filters are not available here); like it, W is a tight frame with W^-1 = W^T.
// One analysis level along an axis of length M:
//   a[k] = sum_n h[n] x[(2k + n) mod M],  d[k] = sum_n g[n] x[(2k + n) mod M],
// with h = (1 + s3, 3 + s3, 3 - s3, 1 - s3) / (4 sqrt 2), s3 = sqrt 3, g[n] = (-1)^n h[3 - n].
#include <algorithm>
#include <cmath>
#include <vector>

#include "pat_internal.cuh"

namespace pat {
namespace {

// Daubechies' 4-tap filters (closed form)
__device__ __forceinline__ float wav_h(int n) {
    const float s3 = 1.7320508075688772f, c = 0.17677669529663688f;   // 1 / (4 sqrt 2)
    return n == 0 ? (1.f + s3) * c : n == 1 ? (3.f + s3) * c : n == 2 ? (3.f - s3) * c : (1.f - s3) * c;
}
__device__ __forceinline__ float wav_g(int n) { return (n & 1 ? -1.f : 1.f) * wav_h(3 - n); }
__device__ __forceinline__ float wav_f(bool high, int n) { return high ? wav_g(n) : wav_h(n); }

// out (M x M block, stride so) = one analysis level of in (M x M block, stride si)
// and, if ll is not NULL, its LL quadrant again into ll (stride M / 2): the next level's input
__global__ void k_wav_analysis(const float* __restrict__ in, int si, float* __restrict__ out, int so, int M,
                               const int* stop, long long ps, float* __restrict__ ll) {
    const long long po = ps * blockIdx.z;   // problem blockIdx.z of a batch: its buffers lie po bytes on
    in = at_bytes(in, po);
    out = at_bytes(out, po);
    ll = ll ? at_bytes(ll, po) : ll;
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= M || y >= M) return;
    const int h2 = M >> 1;
    const bool hx = x >= h2, hy = y >= h2;
    const int kx = hx ? x - h2 : x, ky = hy ? y - h2 : y;
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int yy = (2 * ky + a) % M;
        float row = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) row = fmaf(wav_f(hx, b), __ldg(in + (size_t)yy * si + (2 * kx + b) % M), row);
        acc = fmaf(wav_f(hy, a), row, acc);
    }
    out[(size_t)y * so + x] = acc;
    if (ll && !hx && !hy) ll[(size_t)y * h2 + x] = acc;
}

// out (M x M, stride so) = the transpose of one analysis level applied to the coefficient
// block whose LL quadrant is in ll (stride sl) and whose detail quadrants are in in (stride
// si): out[y][x] = sum over the four quadrants and the taps that reach (y, x) of
// f_y[y - 2k] f_x[x - 2m] c[k][m] (indices mod M).
__global__ void k_wav_synthesis(const float* __restrict__ ll, int sl, const float* __restrict__ in, int si,
                                float* __restrict__ out, int so, int M, const int* stop, long long ps) {
    const long long po = ps * blockIdx.z;
    ll = at_bytes(ll, po);
    in = at_bytes(in, po);
    out = at_bytes(out, po);
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= M || y >= M) return;
    const int h2 = M >> 1;
    float acc = 0.f;
#pragma unroll
    for (int ta = 0; ta < 2; ++ta) {
        const int a = (y & 1) + 2 * ta;                       // tap index along y
        const int ky = ((y - a + M) % M) >> 1;                // coefficient row (y - a is even)
#pragma unroll
        for (int tb = 0; tb < 2; ++tb) {
            const int b = (x & 1) + 2 * tb;
            const int kx = ((x - b + M) % M) >> 1;
            const float cll = __ldg(ll + (size_t)ky * sl + kx), hl = __ldg(in + (size_t)ky * si + kx + h2);
            const float lh = __ldg(in + (size_t)(ky + h2) * si + kx), hh = __ldg(in + (size_t)(ky + h2) * si + kx + h2);
            const float hya = wav_h(a), gya = wav_g(a), hxb = wav_h(b), gxb = wav_g(b);
            acc += hya * (hxb * cll + gxb * hl) + gya * (hxb * lh + gxb * hh);
        }
    }
    out[(size_t)y * so + x] = acc;
}

// r <- clip(r + sigma_r / s * W ubar, -alpha, alpha): the prox of F2* for the scalar
// coefficients of the wavelet model (Sec. 3.2)
__global__ void k_wav_dual(float* __restrict__ r, const float* __restrict__ wub, const float* __restrict__ sig_r,
                           const float* step_mul, const float* scal, long long nn, const int* stop, long long ps) {
    const long long po = ps * blockIdx.y;
    r = at_bytes(r, po);
    wub = at_bytes(wub, po);
    sig_r = at_bytes(sig_r, po);
    step_mul = at_bytes(step_mul, po);
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const float alpha = *at_bytes(scal, po);
    const float v = r[i] + __ldg(sig_r + i) * __ldg(step_mul + 1) * wub[i];
    r[i] = fminf(fmaxf(v, -alpha), alpha);
}

__global__ void k_wav_primal(WavPrimalArgs a, long long ps) {
    const long long po = ps * blockIdx.z;   // every pointer of a is in the problem's workspace
    a.tau_u = at_bytes(a.tau_u, po);
    a.step_mul = at_bytes(a.step_mul, po);
    a.scal = at_bytes(a.scal, po);
    a.kt.acc = at_bytes(a.kt.acc, po);
    a.kt.ymax_bits = at_bytes(a.kt.ymax_bits, po);
    a.kt.tile_kmax = at_bytes(a.kt.tile_kmax, po);
    a.wtr = at_bytes(a.wtr, po);
    a.u = at_bytes(a.u, po);
    if (a.u_old) a.u_old = at_bytes(a.u_old, po);
    a.ubar = at_bytes(a.ubar, po);
    a.kt_clear = at_bytes(a.kt_clear, po);
    a.qmax_next = at_bytes(a.qmax_next, po);
    if (a.stop) a.stop = at_bytes(a.stop, po);
    if (a.iter) a.iter = at_bytes(a.iter, po);
    if (a.stop && *(volatile const int*)a.stop) return;
    const int N = a.n;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        if (a.iter) *a.iter += 1;
        *a.qmax_next = 0u;
    }
    if (gx >= N || gy >= N) return;
    const int gi = gy * N + gx;
    const float uo = a.u[gi];
    if (a.u_old) a.u_old[gi] = uo;
    const float un = uo - __ldg(a.tau_u + gi) * __ldg(a.step_mul) * (a.kt.at(gx, gy, N) + __ldg(a.wtr + gi));
    const float ub = un + __ldg(a.scal + 1) * (un - uo);
    a.u[gi] = un;
    a.ubar[gi] = ub;
    a.kt_clear[gi] = 0;
}

// per-block sums, in the layout of the gap's pixel pass: {|W u|_1, 0, |K^T q + W^T r|_1, 0,
// |u - u_old|^2, |u_old|^2, 0}
__global__ void __launch_bounds__(256) k_wav_gap_pixels(WavGapArgs a, long long ps) {
    const long long po = ps * blockIdx.y;
    a.wu = at_bytes(a.wu, po);
    a.kt.acc = at_bytes(a.kt.acc, po);
    a.kt.ymax_bits = at_bytes(a.kt.ymax_bits, po);
    a.kt.tile_kmax = at_bytes(a.kt.tile_kmax, po);
    a.wtr = at_bytes(a.wtr, po);
    a.u = at_bytes(a.u, po);
    if (a.u_old) a.u_old = at_bytes(a.u_old, po);
    a.partials = at_bytes(a.partials, po);
    if (a.stop) a.stop = at_bytes(a.stop, po);
    if (a.stop && *(volatile const int*)a.stop) return;
    const int N = a.n;
    const long long NN = (long long)N * N;
    float t0 = 0.f, t2 = 0.f, t4 = 0.f, t5 = 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < NN; p += (long long)gridDim.x * blockDim.x) {
        const int gx = (int)(p % N), gy = (int)(p / N);
        t0 += fabsf(a.wu[p]);
        t2 += fabsf(a.kt.at(gx, gy, N) + a.wtr[p]);
        if (a.u_old) {
            const float d = a.u[p] - a.u_old[p];
            t4 += d * d;
            t5 += a.u_old[p] * a.u_old[p];
        }
    }
    double v[4] = {(double)t0, (double)t2, (double)t4, (double)t5};
    __shared__ double sh[4][8];
    for (int c = 0; c < 4; ++c) {
        double x = v[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        v[c] = x;
    }
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 4; ++c) sh[c][threadIdx.x >> 5] = v[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int c = 0; c < 4; ++c) s[c] += sh[c][w];
        double* o = a.partials + (size_t)a.terms * blockIdx.x;
        for (int c = 0; c < a.terms; ++c) o[c] = 0.0;
        o[0] = s[0];
        o[2] = s[1];
        o[4] = s[2];
        o[5] = s[3];
    }
}

__global__ void k_wav_tau(const float* __restrict__ kcol, const double* __restrict__ wcol, float* __restrict__ tau,
                          long long nn) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double s = (double)kcol[i] + wcol[i];
    tau[i] = s > 0 ? (float)(1.0 / s) : 1.f;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
bool wav_levels_ok(int n, int levels) { return levels >= 1 && levels <= 12 && n % (1 << levels) == 0 && (n >> levels) >= 1; }

// Row sums (per coefficient, Mallat layout) and column sums (per pixel) of |W| in FP64.
// W is separable: every 2-D basis function is the product of two 1-D level-l functions,
// so both sums factorise into 1-D sums.  The 1-D level operators are built row by row:
// a row of level l is sum_t f[t] (row (2k + t) mod M of level l - 1's low-pass rows).
void wav_abs_sums(int n, int levels, std::vector<double>& rows, std::vector<double>& cols) {
    const double s3 = std::sqrt(3.0), c = 1.0 / (4.0 * std::sqrt(2.0));
    const double h[4] = {(1 + s3) * c, (3 + s3) * c, (3 - s3) * c, (1 - s3) * c};
    double g[4];
    for (int t = 0; t < 4; ++t) g[t] = ((t & 1) ? -1.0 : 1.0) * h[3 - t];
    rows.assign((size_t)n * n, 0.0);
    cols.assign((size_t)n * n, 0.0);
    std::vector<double> low((size_t)n * n, 0.0);   // current low-pass rows (M rows of length n)
    for (int i = 0; i < n; ++i) low[(size_t)i * n + i] = 1.0;
    int M = n;
    for (int l = 0; l < levels; ++l) {
        const int h2 = M / 2;
        std::vector<double> lo((size_t)h2 * n, 0.0), hi((size_t)h2 * n, 0.0);
        for (int k = 0; k < h2; ++k)
            for (int t = 0; t < 4; ++t) {
                const double* src = &low[(size_t)((2 * k + t) % M) * n];
                for (int x = 0; x < n; ++x) {
                    lo[(size_t)k * n + x] += h[t] * src[x];
                    hi[(size_t)k * n + x] += g[t] * src[x];
                }
            }
        std::vector<double> rl(h2, 0.0), rh(h2, 0.0), cl(n, 0.0), ch(n, 0.0);
        for (int k = 0; k < h2; ++k)
            for (int x = 0; x < n; ++x) {
                rl[k] += std::fabs(lo[(size_t)k * n + x]);
                rh[k] += std::fabs(hi[(size_t)k * n + x]);
                cl[x] += std::fabs(lo[(size_t)k * n + x]);
                ch[x] += std::fabs(hi[(size_t)k * n + x]);
            }
        const bool last = l == levels - 1;
        for (int y = 0; y < h2; ++y)
            for (int x = 0; x < h2; ++x) {
                rows[(size_t)y * n + x + h2] = rl[y] * rh[x];          // HL
                rows[(size_t)(y + h2) * n + x] = rh[y] * rl[x];        // LH
                rows[(size_t)(y + h2) * n + x + h2] = rh[y] * rh[x];   // HH
                if (last) rows[(size_t)y * n + x] = rl[y] * rl[x];     // LL
            }
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x)
                cols[(size_t)y * n + x] += cl[y] * ch[x] + ch[y] * cl[x] + ch[y] * ch[x] + (last ? cl[y] * cl[x] : 0.0);
        low.swap(lo);
        M = h2;
    }
}

// In the launches below, B problems whose buffers lie ps bytes apart (one workspace block
// per problem) run in one grid: the problem index is the grid's last dimension.
static dim3 block_grid(int M, int B) { return dim3(ceil_div(M, 32), ceil_div(M, 8), B); }

// The LL block a level passes to the next lives in scratch, so no level overwrites its own
// input: level l >= 2 reads X_l = scratch for even l and scratch + (N/2)^2 for odd l.
static float* wav_ll_buffer(float* scratch, int N, int l) {
    return (l & 1) ? scratch + (size_t)(N / 2) * (N / 2) : scratch;
}

// out = W in.  scratch: N*N floats.
int launch_wav_analysis(const float* in, int N, int levels, float* out, float* scratch, const int* stop,
                        cudaStream_t st, int B, long long ps) {
    const dim3 blk(32, 8);
    k_wav_analysis<<<block_grid(N, B), blk, 0, st>>>(in, N, out, N, N, stop, ps,
                                                     levels >= 2 ? wav_ll_buffer(scratch, N, 2) : nullptr);
    PAT_LAUNCH_CHECK("k_wav_analysis");
    for (int l = 2, M = N / 2; l <= levels; ++l, M /= 2) {
        k_wav_analysis<<<block_grid(M, B), blk, 0, st>>>(wav_ll_buffer(scratch, N, l), M, out, N, M, stop, ps,
                                                         l < levels ? wav_ll_buffer(scratch, N, l + 1) : nullptr);
        PAT_LAUNCH_CHECK("k_wav_analysis");
    }
    return PAT_OK;
}

// out = W^T in (in is not modified).  scratch: N*N floats; out may not alias in.  Level
// l >= 2 writes its M x M block (M = N >> (l - 1)) into X_l, the next finer level's LL.
int launch_wav_synthesis(const float* in, int N, int levels, float* out, float* scratch, const int* stop,
                         cudaStream_t st, int B, long long ps) {
    const dim3 blk(32, 8);
    const float* ll = in;   // the coarsest level's LL is in the coefficients themselves
    int sl = N;
    for (int l = levels; l >= 1; --l) {
        const int M = N >> (l - 1);
        float* dst = l == 1 ? out : wav_ll_buffer(scratch, N, l);
        k_wav_synthesis<<<block_grid(M, B), blk, 0, st>>>(ll, sl, in, N, dst, l == 1 ? N : M, M, stop, ps);
        PAT_LAUNCH_CHECK("k_wav_synthesis");
        ll = dst;
        sl = M;
    }
    return PAT_OK;
}

int launch_wav_dual(float* r, const float* wub, const float* sig_r, const float* step_mul, const float* scal,
                    long long nn, const int* stop, cudaStream_t st, int B, long long ps) {
    k_wav_dual<<<dim3((unsigned)ceil_div(nn, 256), B), 256, 0, st>>>(r, wub, sig_r, step_mul, scal, nn, stop, ps);
    PAT_LAUNCH_CHECK("k_wav_dual");
    return PAT_OK;
}

int launch_wav_primal(const WavPrimalArgs& a, cudaStream_t st, int B, long long ps) {
    k_wav_primal<<<dim3(ceil_div(a.n, 32), ceil_div(a.n, 8), B), dim3(32, 8), 0, st>>>(a, ps);
    PAT_LAUNCH_CHECK("k_wav_primal");
    return PAT_OK;
}

int launch_wav_gap_pixels(const WavGapArgs& a, int nblocks, cudaStream_t st, int B, long long ps) {
    k_wav_gap_pixels<<<dim3(nblocks, B), 256, 0, st>>>(a, ps);
    PAT_LAUNCH_CHECK("k_wav_gap_pixels");
    return PAT_OK;
}

int launch_wav_tau(const float* kcol, const double* wcol, float* tau, long long nn, cudaStream_t st) {
    k_wav_tau<<<(unsigned)ceil_div(nn, 256), 256, 0, st>>>(kcol, wcol, tau, nn);
    PAT_LAUNCH_CHECK("k_wav_tau");
    return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" int pat_wavelet_transform(int n, int levels, const float* in_dev, float* out_dev, int inverse,
                                     void* stream) {
    if (!in_dev || !out_dev || in_dev == out_dev || n < 2 || !wav_levels_ok(n, levels))
        return fail(PAT_ERR_INVALID_ARG,
                    "pat_wavelet_transform: distinct non-NULL buffers and n divisible by 2^levels (1..12 levels)");
    cudaStream_t st = (cudaStream_t)stream;
    float* scratch = nullptr;
    PAT_CUDA(cudaMallocAsync(&scratch, (size_t)n * n * sizeof(float), st));
    const int rc = inverse ? launch_wav_synthesis(in_dev, n, levels, out_dev, scratch, nullptr, st, 1, 0)
                           : launch_wav_analysis(in_dev, n, levels, out_dev, scratch, nullptr, st, 1, 0);
    cudaFreeAsync(scratch, st);
    return rc;
}
