// The dual-tree complex wavelet transform of the wavelet model (Sec. 2.2, eq. (min_wav);
// Kingsbury's dual tree), its transpose, the |W| sums of the diagonal steps and the
// pointwise kernels of the PDHG that use it (Algorithm 1 with grad -> W, div -> -W^T).
//
// Trees and layout.  Two real orthonormal filter banks, tree a and tree b.  Level 1 uses one
// filter pair in both trees with tree b's input index offset by one sample; levels >= 2 use
// a Q-shift pair: tree b's filters are tree a's reversed in time.  The 2-D transform is four
// separable orthonormal transforms T_t, t = 2 p + q (p: tree along x, q: tree along y; aa,
// ab, ba, bb), each with J levels in the Mallat layout of an N x N plane.  One analysis
// step along an axis of length M with filters (h, g) and offset o:
//   a[k] = sum_n h[n] x[(2k + n + o) mod M],  d[k] = sum_n g[n] x[(2k + n + o) mod M].
// The kernels keep the four tree planes unscaled ("T planes", plane t at offset t N^2).
// W u (4 N^2 values, four planes) is (1/2) T u followed, at every detail position, by the
// orthogonal change to two complex coefficients
//   z1 = ((aa - bb) + i (ab + ba)) / sqrt 2,  z2 = ((aa + bb) + i (ba - ab)) / sqrt 2,
// stored as (Re z1, Im z1, Re z2, Im z2); at the LL positions of level J plane c holds
// (1/2) tree c's coefficient.  Each tree is orthonormal and the change orthogonal, so W is a
// tight frame: W^T W = I, ||W|| = 1.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pat_internal.cuh"

namespace pat {
namespace {

constexpr float kHalfInvSqrt2 = 0.35355339059327373f;   // 1 / (2 sqrt 2)

__device__ __forceinline__ int imod(int a, int m) {
    const int r = a % m;
    return r < 0 ? r + m : r;
}

// filters of tree `tree` (0 = a, 1 = b) at a level: low-pass h, high-pass g, length, offset
struct AxisF {
    const float* h;
    const float* g;
    int len, off;
};
__device__ __forceinline__ AxisF axis_filters(const CwtBank& b, int tree, bool level1) {
    if (level1) return AxisF{b.h1, b.g1, b.l1, tree};
    return tree ? AxisF{b.hb, b.gb, b.lq, 0} : AxisF{b.ha, b.ga, b.lq, 0};
}

// In every kernel below, B problems whose buffers lie pb bytes apart (one workspace block per
// problem) can share one grid: blockIdx.z = 4 b + t for the per-tree kernels (tree t of
// problem b), blockIdx.z = b or blockIdx.y = b for the others.

// One analysis level of the four trees: out plane t (stride so, plane stride ps) block
// M x M from in (plane t at in + t * in_ps, stride si; in_ps = 0 reads one image for all).
__global__ void k_cwt_analysis(const float* __restrict__ in, long long in_ps, int si, float* __restrict__ out,
                               long long ps, int so, int M, int level1, const CwtBank bank, const int* stop,
                               long long pb, float* __restrict__ ll, long long ll_ps) {
    const long long po = pb * (blockIdx.z >> 2);
    in = at_bytes(in, po);
    out = at_bytes(out, po);
    ll = ll ? at_bytes(ll, po) : ll;
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, t = blockIdx.z & 3;
    if (x >= M || y >= M) return;
    const AxisF fx = axis_filters(bank, t >> 1, level1), fy = axis_filters(bank, t & 1, level1);
    const int h2 = M >> 1;
    const bool hx = x >= h2, hy = y >= h2;
    const int kx = hx ? x - h2 : x, ky = hy ? y - h2 : y;
    const float* fxv = hx ? fx.g : fx.h;
    const float* fyv = hy ? fy.g : fy.h;
    const float* src = in + in_ps * t;
    float acc = 0.f;
    for (int a = 0; a < fy.len; ++a) {
        const float* row = src + (size_t)imod(2 * ky + a + fy.off, M) * si;
        float r = 0.f;
        for (int b = 0; b < fx.len; ++b) r = fmaf(fxv[b], __ldg(row + imod(2 * kx + b + fx.off, M)), r);
        acc = fmaf(fyv[a], r, acc);
    }
    out[ps * t + (size_t)y * so + x] = acc;
    if (ll && !hx && !hy) ll[ll_ps * t + (size_t)y * h2 + x] = acc;   // the next level's input (stride M / 2)
}

// Transpose of one analysis level of tree t applied to the coefficient block (in plane t,
// stride si, quadrants of size M/2): value at (y, x) of the M x M output.
// The LL quadrant comes from ll (stride sl) and the three detail quadrants from c (stride
// si); both are c itself for the coarsest level.
__device__ __forceinline__ float cwt_synth_at(const float* __restrict__ ll, int sl, const float* __restrict__ c,
                                              int si, int M, int x, int y, const AxisF& fx, const AxisF& fy) {
    const int h2 = M >> 1;
    float acc = 0.f;
    // taps a with y = 2 ky + a + off (mod M): a has the parity of y - off
    for (int a = imod(y - fy.off, 2); a < fy.len; a += 2) {
        const int ky = imod(y - a - fy.off, M) >> 1;
        float lo = 0.f, hi = 0.f;
        for (int b = imod(x - fx.off, 2); b < fx.len; b += 2) {
            const int kx = imod(x - b - fx.off, M) >> 1;
            const float* r0 = c + (size_t)ky * si;
            const float* r1 = c + (size_t)(ky + h2) * si;
            lo = fmaf(fx.h[b], __ldg(ll + (size_t)ky * sl + kx), fmaf(fx.g[b], __ldg(r0 + kx + h2), lo));
            hi = fmaf(fx.h[b], __ldg(r1 + kx), fmaf(fx.g[b], __ldg(r1 + kx + h2), hi));
        }
        acc = fmaf(fy.h[a], lo, fmaf(fy.g[a], hi, acc));
    }
    return acc;
}

// Levels >= 2: out plane t (M x M, stride so, plane stride ops) from the detail quadrants
// of in plane t (stride si, plane stride ips) and the LL quadrant in ll (stride sl, plane
// stride lps: the level above's output, or in itself at the coarsest level).
__global__ void k_cwt_synthesis(const float* __restrict__ ll, long long lps, int sl, const float* __restrict__ in,
                                long long ips, int si, float* __restrict__ out, long long ops, int so, int M,
                                const CwtBank bank, const int* stop, long long pb) {
    const long long po = pb * (blockIdx.z >> 2);
    ll = at_bytes(ll, po);
    in = at_bytes(in, po);
    out = at_bytes(out, po);
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, t = blockIdx.z & 3;
    if (x >= M || y >= M) return;
    const AxisF fx = axis_filters(bank, t >> 1, false), fy = axis_filters(bank, t & 1, false);
    out[ops * t + (size_t)y * so + x] = cwt_synth_at(ll + lps * t, sl, in + ips * t, si, M, x, y, fx, fy);
}

// Level 1 and the sum of the four trees: out (N x N) = sum_t T_t^T level 1 of plane t (LL
// quadrants from ll, stride sl, plane stride lps).
__global__ void k_cwt_synthesis_sum(const float* __restrict__ ll, long long lps, int sl, const float* __restrict__ in,
                                    long long ips, int si, float* __restrict__ out, int N, const CwtBank bank,
                                    const int* stop, long long pb) {
    const long long po = pb * blockIdx.z;
    ll = at_bytes(ll, po);
    in = at_bytes(in, po);
    out = at_bytes(out, po);
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= N || y >= N) return;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        acc += cwt_synth_at(ll + lps * t, sl, in + ips * t, si, N, x, y, axis_filters(bank, t >> 1, true),
                            axis_filters(bank, t & 1, true));
    out[(size_t)y * N + x] = acc;
}


// The four W-coefficients at one position from the T planes (each times 1/2).
__device__ __forceinline__ void combine_at(const float* __restrict__ T, long long NN, long long i, bool ll, float c[4]) {
    const float aa = __ldg(T + i), ab = __ldg(T + NN + i), ba = __ldg(T + 2 * NN + i), bb = __ldg(T + 3 * NN + i);
    if (ll) {
        c[0] = 0.5f * aa;
        c[1] = 0.5f * ab;
        c[2] = 0.5f * ba;
        c[3] = 0.5f * bb;
    } else {
        c[0] = (aa - bb) * kHalfInvSqrt2;
        c[1] = (ab + ba) * kHalfInvSqrt2;
        c[2] = (aa + bb) * kHalfInvSqrt2;
        c[3] = (ba - ab) * kHalfInvSqrt2;
    }
}

// r <- prox_{sigma F2*}(r + sigma W ubar) (Sec. 3.2) from the T planes of ubar: every complex
// detail coefficient onto the disc of radius alpha (its two rows share one step), every LL
// coefficient clipped to [-alpha, alpha].
__global__ void k_cwt_dual(float* __restrict__ r, const float* __restrict__ T, const float* __restrict__ sig_r,
                           const float* step_mul, const float* scal, int N, int ll_side, const int* stop,
                           long long pb) {
    const long long po = pb * blockIdx.y;
    r = at_bytes(r, po);
    T = at_bytes(T, po);
    sig_r = at_bytes(sig_r, po);
    step_mul = at_bytes(step_mul, po);
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const long long NN = (long long)N * N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NN) return;
    const float alpha = *at_bytes(scal, po);
    const int x = (int)(i % N), y = (int)(i / N);
    const bool ll = x < ll_side && y < ll_side;
    float c[4];
    combine_at(T, NN, i, ll, c);
    const float sm = __ldg(step_mul + 1);
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = fmaf(__ldg(sig_r + k * NN + i) * sm, c[k], r[k * NN + i]);
    if (ll) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = fminf(fmaxf(v[k], -alpha), alpha);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k += 2) {
            const float m2 = __fadd_rn(__fmul_rn(v[k], v[k]), __fmul_rn(v[k + 1], v[k + 1]));
            if (m2 > alpha * alpha) {
                const float sc = alpha * rsqrtf(m2);
                v[k] *= sc;
                v[k + 1] *= sc;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k * NN + i] = v[k];
}

// T planes of W^T: the coefficients r in tree form, each times 1/2 (the change back from the
// complex pairs is the transpose of the change above)
__global__ void k_cwt_uncombine(const float* __restrict__ r, float* __restrict__ T, int N, int ll_side, const int* stop,
                                long long pb) {
    const long long po = pb * blockIdx.y;
    r = at_bytes(r, po);
    T = at_bytes(T, po);
    stop = stop ? at_bytes(stop, po) : stop;
    if (stop && *(volatile const int*)stop) return;
    const long long NN = (long long)N * N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NN) return;
    const int x = (int)(i % N), y = (int)(i / N);
    const float c0 = r[i], c1 = r[NN + i], c2 = r[2 * NN + i], c3 = r[3 * NN + i];
    if (x < ll_side && y < ll_side) {
        T[i] = 0.5f * c0;
        T[NN + i] = 0.5f * c1;
        T[2 * NN + i] = 0.5f * c2;
        T[3 * NN + i] = 0.5f * c3;
    } else {
        T[i] = (c0 + c2) * kHalfInvSqrt2;
        T[NN + i] = (c1 - c3) * kHalfInvSqrt2;
        T[2 * NN + i] = (c1 + c3) * kHalfInvSqrt2;
        T[3 * NN + i] = (c2 - c0) * kHalfInvSqrt2;
    }
}

// per-block sums in the layout of the gap's pixel pass: {||W u||_1, 0, |K^T q + W^T r|_1, 0,
// |u - u_old|^2, |u_old|^2, 0}; W u from the T planes of u
__global__ void __launch_bounds__(256) k_cwt_gap_pixels(CwtGapArgs a, long long pb) {
    const long long po = pb * blockIdx.y;
    a.tu = at_bytes(a.tu, po);
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
        const bool ll = gx < a.ll_side && gy < a.ll_side;
        float c[4];
        combine_at(a.tu, NN, p, ll, c);
        t0 += ll ? fabsf(c[0]) + fabsf(c[1]) + fabsf(c[2]) + fabsf(c[3])
                 : sqrtf(c[0] * c[0] + c[1] * c[1]) + sqrtf(c[2] * c[2] + c[3] * c[3]);
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

dim3 grid_of(int M, int z) { return dim3(ceil_div(M, 32), ceil_div(M, 8), z); }

}  // namespace

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

// The filter bank from the level-1 low-pass h1 and the Q-shift low-pass hq of tree a (FP64
// on the host): high-pass g[n] = (-1)^n h[L - 1 - n]; tree b's Q-shift filters are tree a's
// reversed.  NULL selects the closed-form defaults: Daubechies' 4-tap filter
// (1 + s3, 3 + s3, 3 - s3, 1 - s3) / (4 sqrt 2) at level 1, and the orthonormal 4-tap filter
// (5 - s15, 5 + s15, 3 + s15, 3 - s15) / (8 sqrt 2) (centre 1.25, a quarter sample before
// its midpoint) at levels >= 2.  Each filter must be orthonormal (sum h^2 = 1, even shifts
// orthogonal, sum h = sqrt 2, to 1e-6), of even length 2..16.
int cwt_bank(const double* h1, int l1, const double* hq, int lq, CwtBank& bank, std::vector<double>* h1_out,
             std::vector<double>* hq_out) {
    const double s3 = std::sqrt(3.0), s15 = std::sqrt(15.0);
    const double d4[4] = {(1 + s3) / (4 * std::sqrt(2.0)), (3 + s3) / (4 * std::sqrt(2.0)),
                          (3 - s3) / (4 * std::sqrt(2.0)), (1 - s3) / (4 * std::sqrt(2.0))};
    const double q4[4] = {(5 - s15) / (8 * std::sqrt(2.0)), (5 + s15) / (8 * std::sqrt(2.0)),
                          (3 + s15) / (8 * std::sqrt(2.0)), (3 - s15) / (8 * std::sqrt(2.0))};
    std::vector<double> a(h1 ? h1 : d4, h1 ? h1 + l1 : d4 + 4), q(hq ? hq : q4, hq ? hq + lq : q4 + 4);
    for (const std::vector<double>* f : {&a, &q}) {
        const int L = (int)f->size();
        if (L < 2 || L > CWT_MAX_TAPS || (L & 1))
            return fail(PAT_ERR_INVALID_ARG, "DT-CWT filters: even length 2..16 needed");
        double s = 0.0;
        for (double v : *f) s += v;
        if (std::fabs(s - std::sqrt(2.0)) > 1e-6) return fail(PAT_ERR_INVALID_ARG, "DT-CWT filters: sum must be sqrt 2");
        for (int k = 0; 2 * k < L; ++k) {
            double d = 0.0;
            for (int n = 0; n + 2 * k < L; ++n) d += (*f)[n] * (*f)[n + 2 * k];
            if (std::fabs(d - (k == 0 ? 1.0 : 0.0)) > 1e-6)
                return fail(PAT_ERR_INVALID_ARG, "DT-CWT filters: not orthonormal (sum h[n] h[n + 2k] != delta_k)");
        }
    }
    auto hp = [](const std::vector<double>& h, int n) {
        const int L = (int)h.size();
        return ((n & 1) ? -1.0 : 1.0) * h[L - 1 - n];
    };
    bank = CwtBank{};
    bank.l1 = (int)a.size();
    bank.lq = (int)q.size();
    for (int n = 0; n < bank.l1; ++n) {
        bank.h1[n] = (float)a[n];
        bank.g1[n] = (float)hp(a, n);
    }
    std::vector<double> qb(q.rbegin(), q.rend());
    for (int n = 0; n < bank.lq; ++n) {
        bank.ha[n] = (float)q[n];
        bank.ga[n] = (float)hp(q, n);
        bank.hb[n] = (float)qb[n];
        bank.gb[n] = (float)hp(qb, n);
    }
    if (h1_out) *h1_out = a;
    if (hq_out) *hq_out = q;
    return PAT_OK;
}

// Row sums (4 N^2, the W layout) and column sums (N^2) of |W| in FP64.  Every row of W is a
// circular shift of the row at coefficient index (0, 0) of its level, orientation and
// plane, by 2^l per index, so all rows of one (level, orientation, plane) have the same sum,
// and a column's sum over them is that row's |entries| summed over the pixels congruent to
// the column modulo 2^l.  A row is built from the 1-D level functions of the two trees: the
// level-l functions of a tree are sum_t f[t] (level l - 1 low-pass row (2k + t + o) mod M).
void cwt_abs_sums(int n, int levels, const std::vector<double>& h1, const std::vector<double>& hq,
                  std::vector<double>& rows, std::vector<double>& cols) {
    const size_t NN = (size_t)n * n;
    rows.assign(4 * NN, 0.0);
    cols.assign(NN, 0.0);
    auto hp = [](const std::vector<double>& h) {
        std::vector<double> g(h.size());
        for (size_t k = 0; k < h.size(); ++k) g[k] = ((k & 1) ? -1.0 : 1.0) * h[h.size() - 1 - k];
        return g;
    };
    std::vector<double> qb(hq.rbegin(), hq.rend());
    // low-pass rows of the previous level per tree (M rows of length n)
    std::vector<double> low[2];
    for (int tr = 0; tr < 2; ++tr) {
        low[tr].assign(NN, 0.0);
        for (int i = 0; i < n; ++i) low[tr][(size_t)i * n + i] = 1.0;
    }
    int M = n;
    const double c2 = 1.0 / (2.0 * std::sqrt(2.0));
    std::vector<double> R(NN);
    for (int l = 1; l <= levels; ++l) {
        const int h2 = M / 2;
        std::vector<double> lo[2], hi[2];   // index-0 function and all rows of the new level
        for (int tr = 0; tr < 2; ++tr) {
            const std::vector<double>& h = l == 1 ? h1 : (tr ? qb : hq);
            const std::vector<double> g = hp(h);
            const int off = l == 1 ? tr : 0;
            lo[tr].assign((size_t)h2 * n, 0.0);
            hi[tr].assign((size_t)h2 * n, 0.0);
            for (int k = 0; k < h2; ++k)
                for (size_t t = 0; t < h.size(); ++t) {
                    const double* src = &low[tr][(size_t)((2 * k + (int)t + off) % M) * n];
                    for (int x = 0; x < n; ++x) {
                        lo[tr][(size_t)k * n + x] += h[t] * src[x];
                        hi[tr][(size_t)k * n + x] += g[t] * src[x];
                    }
                }
        }
        const int P = 1 << l;   // period of the column sums of this level
        const bool last = l == levels;
        // orientations: (x high, y high) in {(1,0) HL, (0,1) LH, (1,1) HH}, and LL at the last level
        for (int o = 0; o < (last ? 4 : 3); ++o) {
            const bool xh = o == 0 || o == 2, yh = o == 1 || o == 2, isll = o == 3;
            const double* fx[2] = {(xh ? hi[0] : lo[0]).data(), (xh ? hi[1] : lo[1]).data()};   // index 0 rows
            const double* fy[2] = {(yh ? hi[0] : lo[0]).data(), (yh ? hi[1] : lo[1]).data()};
            const int bx = isll ? 0 : (xh ? h2 : 0), by = isll ? 0 : (yh ? h2 : 0);
            for (int c = 0; c < 4; ++c) {
                // R[y][x] = the (0, 0) row of plane c
                for (int y = 0; y < n; ++y)
                    for (int x = 0; x < n; ++x) {
                        const double aa = fy[0][y] * fx[0][x], ab = fy[1][y] * fx[0][x];
                        const double ba = fy[0][y] * fx[1][x], bb = fy[1][y] * fx[1][x];
                        double v;
                        if (isll) v = 0.5 * (c == 0 ? aa : c == 1 ? ab : c == 2 ? ba : bb);
                        else v = c2 * (c == 0 ? aa - bb : c == 1 ? ab + ba : c == 2 ? aa + bb : ba - ab);
                        R[(size_t)y * n + x] = std::fabs(v);
                    }
                double s = 0.0;
                std::vector<double> fold((size_t)P * P, 0.0);
                for (int y = 0; y < n; ++y)
                    for (int x = 0; x < n; ++x) {
                        s += R[(size_t)y * n + x];
                        fold[(size_t)(y % P) * P + (x % P)] += R[(size_t)y * n + x];
                    }
                for (int ky = 0; ky < h2; ++ky)
                    for (int kx = 0; kx < h2; ++kx) rows[c * NN + (size_t)(by + ky) * n + bx + kx] = s;
                for (int y = 0; y < n; ++y)
                    for (int x = 0; x < n; ++x) cols[(size_t)y * n + x] += fold[(size_t)(y % P) * P + (x % P)];
            }
        }
        low[0].swap(lo[0]);
        low[1].swap(lo[1]);
        M = h2;
    }
}

// The LL block a level passes to the next lives in scratch, so no level overwrites its own
// input: level l >= 2 reads buffer X_l and writes X_{l+1}, X_l = scratch (4 (N/2)^2 floats)
// for even l and scratch + N^2 (4 (N/4)^2 floats) for odd l.  scratch: 5 N^2 / 4 floats.
static float* cwt_ll_buffer(float* scratch, int N, int l) { return (l & 1) ? scratch + (size_t)N * N : scratch; }

// out (4 T planes of N x N) = T in.
int launch_cwt_analysis(const float* in, int N, int levels, const CwtBank& bank, float* out, float* scratch,
                        const int* stop, cudaStream_t st, int B, long long pb) {
    const dim3 blk(32, 8);
    const long long NN = (long long)N * N;
    k_cwt_analysis<<<grid_of(N, 4 * B), blk, 0, st>>>(in, 0, N, out, NN, N, N, 1, bank, stop, pb,
                                                      levels >= 2 ? cwt_ll_buffer(scratch, N, 2) : nullptr,
                                                      (long long)(N / 2) * (N / 2));
    PAT_LAUNCH_CHECK("k_cwt_analysis");
    for (int l = 2, M = N / 2; l <= levels; ++l, M /= 2) {
        const long long mm = (long long)M * M;
        k_cwt_analysis<<<grid_of(M, 4 * B), blk, 0, st>>>(cwt_ll_buffer(scratch, N, l), mm, M, out, NN, N, M, 0, bank,
                                                          stop, pb,
                                                          l < levels ? cwt_ll_buffer(scratch, N, l + 1) : nullptr,
                                                          (long long)(M / 2) * (M / 2));
        PAT_LAUNCH_CHECK("k_cwt_analysis");
    }
    return PAT_OK;
}

// out (N x N) = sum_t T_t^T of the T planes in (not modified).  Level l >= 2 writes its
// M x M block (M = N >> (l - 1)) into X_l, which the next finer level reads as its LL.
int launch_cwt_synthesis(float* in, int N, int levels, const CwtBank& bank, float* out, float* scratch,
                         const int* stop, cudaStream_t st, int B, long long pb) {
    const dim3 blk(32, 8);
    const long long NN = (long long)N * N;
    const float* ll = in;   // the coarsest level's LL is in the planes themselves
    long long lps = NN;
    int sl = N;
    for (int l = levels; l >= 2; --l) {
        const int M = N >> (l - 1);
        const long long mm = (long long)M * M;
        float* dst = cwt_ll_buffer(scratch, N, l);
        k_cwt_synthesis<<<grid_of(M, 4 * B), blk, 0, st>>>(ll, lps, sl, in, NN, N, dst, mm, M, M, bank, stop, pb);
        PAT_LAUNCH_CHECK("k_cwt_synthesis");
        ll = dst;
        lps = mm;
        sl = M;
    }
    k_cwt_synthesis_sum<<<grid_of(N, B), blk, 0, st>>>(ll, lps, sl, in, NN, N, out, N, bank, stop, pb);
    PAT_LAUNCH_CHECK("k_cwt_synthesis_sum");
    return PAT_OK;
}

int launch_cwt_dual(float* r, const float* T, const float* sig_r, const float* step_mul, const float* scal, int N,
                    int levels, const int* stop, cudaStream_t st, int B, long long pb) {
    const long long NN = (long long)N * N;
    k_cwt_dual<<<dim3((unsigned)ceil_div(NN, 256), B), 256, 0, st>>>(r, T, sig_r, step_mul, scal, N, N >> levels,
                                                                     stop, pb);
    PAT_LAUNCH_CHECK("k_cwt_dual");
    return PAT_OK;
}

int launch_cwt_uncombine(const float* r, float* T, int N, int levels, const int* stop, cudaStream_t st, int B,
                         long long pb) {
    const long long NN = (long long)N * N;
    k_cwt_uncombine<<<dim3((unsigned)ceil_div(NN, 256), B), 256, 0, st>>>(r, T, N, N >> levels, stop, pb);
    PAT_LAUNCH_CHECK("k_cwt_uncombine");
    return PAT_OK;
}

int launch_cwt_gap_pixels(const CwtGapArgs& a, int nblocks, cudaStream_t st, int B, long long pb) {
    k_cwt_gap_pixels<<<dim3(nblocks, B), 256, 0, st>>>(a, pb);
    PAT_LAUNCH_CHECK("k_cwt_gap_pixels");
    return PAT_OK;
}

// W in (4 planes) from T planes: the change to complex pairs, written out (for the API)
__global__ void k_cwt_combine(const float* __restrict__ T, float* __restrict__ out, int N, int ll_side) {
    const long long NN = (long long)N * N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NN) return;
    float c[4];
    combine_at(T, NN, i, (int)(i % N) < ll_side && (int)(i / N) < ll_side, c);
    for (int k = 0; k < 4; ++k) out[k * NN + i] = c[k];
}

}  // namespace pat

using namespace pat;

extern "C" int pat_dtcwt_transform(int n, int levels, const double* h1_host, int l1, const double* hq_host, int lq,
                                   const float* in_dev, float* out_dev, int inverse, void* stream) {
    if (!in_dev || !out_dev || in_dev == out_dev || n < 2 || !wav_levels_ok(n, levels))
        return fail(PAT_ERR_INVALID_ARG,
                    "pat_dtcwt_transform: distinct non-NULL buffers and n divisible by 2^levels (1..12 levels)");
    CwtBank bank;
    int rc = cwt_bank(h1_host, l1, hq_host, lq, bank, nullptr, nullptr);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long NN = (long long)n * n;
    float* buf = nullptr;   // 4 T planes + scratch (5 N^2 / 4)
    PAT_CUDA(cudaMallocAsync(&buf, (size_t)(4 * NN + NN + NN / 4) * sizeof(float), st));
    float* T = buf;
    float* scratch = buf + 4 * NN;
    if (inverse) {
        rc = launch_cwt_uncombine(in_dev, T, n, levels, nullptr, st, 1, 0);
        if (!rc) rc = launch_cwt_synthesis(T, n, levels, bank, out_dev, scratch, nullptr, st, 1, 0);
    } else {
        rc = launch_cwt_analysis(in_dev, n, levels, bank, T, scratch, nullptr, st, 1, 0);
        if (!rc) {
            k_cwt_combine<<<(unsigned)ceil_div(NN, 256), 256, 0, st>>>(T, out_dev, n, n >> levels);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = fail(PAT_ERR_CUDA, "k_cwt_combine");
        }
    }
    cudaFreeAsync(buf, st);
    return rc;
}
