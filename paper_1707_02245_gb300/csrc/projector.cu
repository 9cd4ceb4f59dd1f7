// Matrix-free circular-mean projector K and its exact transpose K^T (Sec. 3.3.1,
// Sec. 4.2 eq. (K_def)), plus the fused data-row kernels of the PDHG iteration.
//
// Thread mapping of K: four lanes per data row (d, k), one per angular phase; a warp
// holds 8 consecutive radii of one detector and walks the group's angular window in
// lockstep, so at every step its 32 points form a 4-angle x 8-radius patch of the polar
// grid (neighbouring lanes touch neighbouring pixels).  A block holds adjacent detectors
// at the same radii, whose arcs cross the same pixels, so its warps share L1 lines.  Each
// point is interpolated bilinearly between pixel centres.
//
// The hot path reads a zero-bordered copy of the image ((N+2)^2 floats, pixel (i, j) at
// (j+1)(N+2) + i+1) so a point with taps i0, j0 in [-1, N-1] needs no per-tap test.
#include <algorithm>

#include "pat_internal.cuh"
#include "reduce.cuh"

namespace pat {

template <bool PADDED>
__device__ __forceinline__ float fetch4(const float* __restrict__ u, int N, const Taps& t, float& v10,
                                        float& v01, float& v11) {
    if (PADDED) {
        const int P = N + 2;
        const float* p = u + (t.j0 + 1) * P + (t.i0 + 1);
        v10 = __ldg(p + 1);
        v01 = __ldg(p + P);
        v11 = __ldg(p + P + 1);
        return __ldg(p);
    } else {
        const bool x0 = t.i0 >= 0, x1 = t.i0 + 1 < N, y0 = t.j0 >= 0, y1 = t.j0 + 1 < N;
        const float* p = u + t.j0 * N + t.i0;
        v10 = (x1 && y0) ? __ldg(p + 1) : 0.f;
        v01 = (x0 && y1) ? __ldg(p + N) : 0.f;
        v11 = (x1 && y1) ? __ldg(p + N + 1) : 0.f;
        return (x0 && y0) ? __ldg(p) : 0.f;
    }
}

// Row mapping of the projector kernels: a warp holds KGRP = 8 consecutive radii of one
// detector times NPH = 4 angular phases; lane = ph * 8 + kl.  Phase ph walks the group's
// angular window at m = m_first + ph, + ph + 4, ...  so at every step the warp evaluates
// a 4 (angles) x 8 (radii) patch of the polar grid, which is a compact patch of pixels.
constexpr int NPH = 4;
// unroll factors of the forward's angular loop and of the K^T candidate loop (0: the
// compiler's choice)
#ifndef PAT_FWD_UNROLL
#define PAT_FWD_UNROLL 0
#endif
#ifndef PAT_ADJ_UNROLL
#define PAT_ADJ_UNROLL 0
#endif
#ifndef PAT_ADJ_RADIUS_FMA
#define PAT_ADJ_RADIUS_FMA 1   // K^T evaluates r_k (one FMA) instead of gathering rk[k]
#endif
#if PAT_FWD_UNROLL > 0
constexpr int FWD_UNROLL = PAT_FWD_UNROLL;
#endif
#if PAT_ADJ_UNROLL > 0
constexpr int ADJ_UNROLL = PAT_ADJ_UNROLL;
#endif
// A row block is ROW_WARPS warps: FWD_DW adjacent detectors times FWD_KW groups of 8 radii.
#ifndef PAT_FWD_DW
#define PAT_FWD_DW 8
#endif
#ifndef PAT_FWD_WARPS
#define PAT_FWD_WARPS 16
#endif
constexpr int ROW_WARPS = PAT_FWD_WARPS;
constexpr int FWD_DW = PAT_FWD_DW;
constexpr int FWD_KW = ROW_WARPS / FWD_DW;
static_assert(FWD_DW * FWD_KW == ROW_WARPS, "FWD_DW must divide ROW_WARPS");
constexpr int ROWS_PER_BLOCK = ROW_WARPS * KGRP;
constexpr int ROW_THREADS = ROWS_PER_BLOCK * NPH;
// resident row blocks per SM that the register budget must allow (0: the compiler's choice)
#ifndef PAT_FWD_MIN_BLOCKS
#define PAT_FWD_MIN_BLOCKS 0
#endif
#if PAT_FWD_MIN_BLOCKS > 0
#define PAT_ROW_BOUNDS __launch_bounds__(ROW_THREADS, PAT_FWD_MIN_BLOCKS)
#else
#define PAT_ROW_BOUNDS __launch_bounds__(ROW_THREADS)
#endif

struct RowLane {
    int d, k, ph;
    bool valid;
};

// lane of row block (kb, db): warp w takes detector db FWD_DW + w / FWD_KW and the radii
// group kb FWD_KW + w % FWD_KW; lanes past the last detector or radius are not valid
// (their detector index is clamped so that table reads stay in range)
__device__ __forceinline__ RowLane row_lane(const GeomView& g, int kb, int db) {
    RowLane r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = db * FWD_DW + warp / FWD_KW;
    r.ph = lane >> 3;
    r.k = (kb * FWD_KW + warp % FWD_KW) * KGRP + (lane & 7);
    r.valid = r.k < g.n_t && d < g.n_det;
    r.d = min(d, g.n_det - 1);
    return r;
}

// row blocks along the radii (the grid's other dimension runs over detector groups)
__device__ __forceinline__ int row_blocks(const GeomView& g) {
    return (g.n_t + FWD_KW * KGRP - 1) / (FWD_KW * KGRP);
}

// Partial integral of the bilinear image over circle (d, k) for one angular phase.
// QUAD: u points at the float4 quads (one load per point; layout quad_index); otherwise u is the plain
// N*N image read with per-tap bounds tests.
template <bool QUAD>
__device__ __forceinline__ float circle_partial(const GeomView& g, const float* __restrict__ u, const RowLane& rl) {
    const int2 w = __ldg(&g.win[rl.d * g.n_kgrp + min(rl.k / KGRP, g.n_kgrp - 1)]);
    const float2 det = __ldg(&g.det[rl.d]);
    const float r = rl.valid ? __ldg(&g.rk[rl.k]) : 0.f;
    float acc = 0.f;
    int m = w.x + rl.ph;
    if (m >= g.quad_m) m -= g.quad_m;
#if PAT_FWD_UNROLL > 0
#pragma unroll FWD_UNROLL
#endif
    for (int j = rl.ph; j < w.y; j += NPH) {
        const float2 cs = __ldg(&g.cs[m]);
        m += NPH;
        if (m >= g.quad_m) m -= g.quad_m;
        Taps t;
        if (point_taps(g, det, r, cs, t) && rl.valid) {
            float v00, v10, v01, v11;
            if (QUAD) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(u) + quad_index(t.i0 + 1, t.j0 + 1, g.n));
                v00 = v.x;
                v10 = v.y;
                v01 = v.z;
                v11 = v.w;
            } else {
                v00 = fetch4<false>(u, g.n, t, v10, v01, v11);
            }
            const float a = fmaf(t.ax, v10 - v00, v00);
            const float b = fmaf(t.ax, v11 - v01, v01);
            acc += fmaf(t.ay, b - a, a);
        }
    }
    return acc;
}

// Sum over the four phases (lanes kl, kl+8, kl+16, kl+24); valid in every lane.
__device__ __forceinline__ float phase_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// y = K u
__global__ void PAT_ROW_BOUNDS k_forward(GeomView g, const float* __restrict__ u, float* __restrict__ y) {
    const RowLane rl = row_lane(g, blockIdx.x, blockIdx.y);
    const float s = phase_sum(circle_partial<false>(g, u, rl));
    if (rl.valid && rl.ph == 0) y[(size_t)rl.d * g.n_t + rl.k] = s * __ldg(&g.wk[rl.k]);
}

// q <- prox_{sigma F1*}(q + sigma K ubar) = (q + sigma (K ubar - f)) / (1 + sigma)  (Sec. 3.2)
// for the rows of row block kb of detector d.  Also records q w_k for the K^T that follows
// and max |q| (as float bits) for its fixed-point scale.
__device__ __forceinline__ void forward_prox_rows(const FwdProxArgs& a, int kb, int d) {
    const GeomView& g = a.g;
    const RowLane rl = row_lane(g, kb, d);
    // issued before the circle sums so that its latency overlaps them
    const float smul = a.step_mul ? __ldg(a.step_mul + 1) : 1.f;
    const float s = phase_sum(circle_partial<true>(g, reinterpret_cast<const float*>(a.ubar_quad), rl));
    float aq = 0.f;
    if (rl.valid && rl.ph == 0) {
        const size_t i = (size_t)rl.d * g.n_t + rl.k;
        const float wk = __ldg(&g.wk[rl.k]);
        const float ku = s * wk;
        const float sg = (a.sig_q ? a.sig_q[i] : a.sig_scalar) * smul;
        const float qn = (a.q[i] + sg * (ku - a.f[i])) / (1.f + sg);
        a.q[i] = qn;
        a.qw[i] = qn * wk;
        aq = fabsf(qn);
    }
    // block max of |q| (a NaN's bits compare greater than every finite value's)
    unsigned bits = __float_as_uint(aq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
    __shared__ unsigned wmax[ROW_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = bits;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned m = 0;
        for (int w = 0; w < ROW_THREADS / 32; ++w) m = max(m, wmax[w]);
        if (m) atomicMax(a.qmax_bits, m);
    }
}

__global__ void PAT_ROW_BOUNDS k_forward_prox_b(const FwdProxArgs* __restrict__ args,
                                                               const int2* __restrict__ map) {
    const int2 pm = map[blockIdx.x];
    __shared__ FwdProxArgs sa;
    const FwdProxArgs& a = stage_args(args, pm.x, sa);
    if (a.stop && *(volatile const int*)a.stop) return;
    const int nkb = row_blocks(a.g);
    forward_prox_rows(a, pm.y % nkb, pm.y / nkb);
}

// max |y| over n values as float bits (atomicMax; *out must start at 0)
__global__ void k_absmax(const float* __restrict__ y, long long n, unsigned* __restrict__ out) {
    unsigned m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(y[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// FP64 partial sums for the duality gap over data rows:
//   {sum (K u - f)^2, sum q^2, sum q f}   one triple per (local) block lb
template <bool QUAD>
__device__ __forceinline__ void forward_gap_rows(const FwdGapArgs& a, int kb, int d, int lb) {
    const GeomView& g = a.g;
    const RowLane rl = row_lane(g, kb, d);
    const float* img = QUAD ? reinterpret_cast<const float*>(a.u_quad) : a.u;
    const float s = phase_sum(circle_partial<QUAD>(g, img, rl));
    // per-row terms in FP32; warp sums as FP32 pairs, block sums in FP64 (GB300's FP64 pipe
    // is 1/64 of FP32)
    float t[GAP_DATA_TERMS] = {0.f, 0.f, 0.f, 0.f};
    if (rl.valid && rl.ph == 0) {
        const float ku = s * __ldg(&g.wk[rl.k]);
        const size_t i = (size_t)rl.d * g.n_t + rl.k;
        const float res = ku - a.f[i];
        const float qi = a.q[i];
        t[0] = res * res;
        t[1] = qi * qi;
        t[2] = qi * a.f[i];
        t[3] = fabsf(qi - res);   // dual residual of the data term: q - dF1(Ku)
    }
    double sum[GAP_DATA_TERMS];
    block_sum_pair<GAP_DATA_TERMS>(t, sum);
    if (threadIdx.x == 0)
        for (int c = 0; c < GAP_DATA_TERMS; ++c) a.partials[GAP_DATA_TERMS * lb + c] = sum[c];
}

__global__ void PAT_ROW_BOUNDS k_forward_gap_b(const FwdGapArgs* __restrict__ args,
                                                              const int2* __restrict__ map) {
    const int2 pm = map[blockIdx.x];
    __shared__ FwdGapArgs sa;
    const FwdGapArgs& a = stage_args(args, pm.x, sa);
    if (a.stop && *(volatile const int*)a.stop) return;
    const int nkb = row_blocks(a.g);
    if (a.u_quad)
        forward_gap_rows<true>(a, pm.y % nkb, pm.y / nkb, pm.y);
    else
        forward_gap_rows<false>(a, pm.y % nkb, pm.y / nkb, pm.y);
}

// ---------------------------------------------------------------------------------
// K^T by pixel tiles with exact fixed-point accumulation.
//
// A CTA owns a share of one WTILE x WTILE pixel tile's candidate points.  Its shared
// accumulator (with a one-pixel ring, so every point whose taps touch the tile can add
// all four weights) holds int32 fixed-point values: every pixel satisfies
//   |(K^T y)(p)| <= max|y| * (K^T 1)(p)        (all entries of K are >= 0),
// so with the scale S = 2^30 / (max|y| * max over the ATILE tile of K^T 1) no partial sum
// of a tile pixel exceeds 2^30 and integer addition (native shared atomics, associative,
// hence deterministic) replaces floating-point atomics.  The resolution 2^-30 of that
// bound is finer than FP32 accumulation of the same terms.  Ring cells are dropped.
//
// Work: geometry creation cuts every ray (detector, angle) of a tile's polar box to the
// segment of radii whose points can have taps in the tile, concatenates the segments
// into the tile's candidate list, and cuts the lists into equal work items that fill one
// wave of resident CTAs (see the work-item function below).  Every candidate uses the
// forward projector's FP32 position and tap arithmetic, so the CTA adds exactly the
// entries of K^T that belong to its pixels.  Items of one scale tile share its scale, so
// their fixed-point tiles add exactly (in any order) into one image with integer atomics.
// ---------------------------------------------------------------------------------
#ifndef PAT_ADJ_THREADS
#define PAT_ADJ_THREADS 256
#endif
constexpr int ATHREADS = PAT_ADJ_THREADS;   // threads of a K^T CTA
#ifndef PAT_ADJ_MIN_BLOCKS
#define PAT_ADJ_MIN_BLOCKS 5
#endif
constexpr int ADJ_MIN_BLOCKS = PAT_ADJ_MIN_BLOCKS;   // resident CTAs per SM the register budget allows
// first step of the binary search over an item's segments: a power of two with
// 2 * ASTEP >= ARAYS, so that the halving steps reach every index below ARAYS
constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }
constexpr int ASTEP = pow2_at_least(ARAYS) / 2;
static_assert(2 * ASTEP >= ARAYS && (ASTEP & (ASTEP - 1)) == 0, "binary search steps");


// One work item of K^T: an equal share [c0, c1) of one tile's candidate list (the
// concatenated ray segments the host cut to the tile's tap window).  Thread t takes the
// contiguous run [c0 + t C, c0 + (t + 1) C), C = ceil((c1 - c0) / ATHREADS), so every
// thread has the same number of candidates and lanes that add at the same time sit C
// candidates apart (different pixels).  Each candidate is evaluated with the forward's
// FP32 point arithmetic; one whose taps fall outside the tile window is skipped.
template <bool PREMUL>
__device__ __forceinline__ void adjoint_item(const AdjArgs& a, int item_index) {
    const GeomView& g = a.g;
    const int N = g.n, T = g.n_t;
    const AdjItem* ip = a.items + item_index;
    const int tile = __ldg(&ip->tile), ray0 = __ldg(&ip->ray0), nray = __ldg(&ip->nray);
    const int c0 = __ldg(&ip->c0), c1 = __ldg(&ip->c1);
    const int x0 = (tile % a.wtiles_x) * WTILE, y0 = (tile / a.wtiles_x) * WTILE;
    const int tid = threadIdx.x;
    constexpr int AW = WTILE + 2;
    __shared__ int acc[AW * AW];
    __shared__ int4 s_ray[ARAYS + 1];   // {detector, angle, first k, prefix}
    for (int c = tid; c < AW * AW; c += ATHREADS) acc[c] = 0;
    for (int i = tid; i <= nray; i += ATHREADS) s_ray[i] = __ldg(&a.rays[ray0 + i]);
    // the scale of the ATILE tile that holds this work tile
    const float bound = __uint_as_float(*a.ymax_bits) * __ldg(&a.tile_kmax[(y0 / ATILE) * a.tiles_x + x0 / ATILE]);
    const float scale = 1073741824.0f / bound;  // 2^30 / bound
#if PAT_ADJ_RADIUS_FMA
    const float dr_f = g.dr_f, rh_f = g.rh_f;
#else
    const float* __restrict__ rk = g.rk;
#endif
    const float* __restrict__ wk = g.wk;
    const float* __restrict__ y = a.y;
    __syncthreads();

    if (bound > 0.f && isfinite(bound) && nray > 0) {
        const int C = (c1 - c0 + ATHREADS - 1) / ATHREADS;
        int p = c0 + tid * C;
        const int p_end = min(c1, p + C);
        if (p < p_end) {
            int j = 0;  // last segment whose prefix is <= p (the one holding p)
#pragma unroll
            for (int step = ASTEP; step > 0; step >>= 1)
                if (j + step < nray && s_ray[j + step].w <= p) j += step;
            // one flat loop over the run: a segment change is a short branch, so the lanes
            // of a warp stay converged on the point arithmetic
            int4 ray = s_ray[j];
            int seg_end = s_ray[j + 1].w;
            float2 det = __ldg(&g.det[ray.x]);
            float2 cs = __ldg(&g.cs[ray.y]);
            const float* __restrict__ yrow = y + (size_t)ray.x * T;
            int k = ray.z + (p - ray.w);
#if PAT_ADJ_UNROLL > 0
#pragma unroll ADJ_UNROLL
#endif
            for (; p < p_end; ++p, ++k) {
                if (p == seg_end) {  // segments are never empty
                    ++j;
                    ray = s_ray[j];
                    seg_end = s_ray[j + 1].w;
                    det = __ldg(&g.det[ray.x]);
                    cs = __ldg(&g.cs[ray.y]);
                    yrow = y + (size_t)ray.x * T;
                    k = ray.z;
                }
                Taps t;
#if PAT_ADJ_RADIUS_FMA
                point_coords(g, det, radius(k, dr_f, rh_f), cs, t);   // = rk[k], bit for bit
#else
                point_coords(g, det, __ldg(&rk[k]), cs, t);
#endif
                // taps in the tile window (ring cells off the tile are dropped later)
                const int li = t.i0 - x0 + 1, lj = t.j0 - y0 + 1;
                if ((unsigned)li > (unsigned)WTILE || (unsigned)lj > (unsigned)WTILE) continue;
                const float c = (PREMUL ? __ldg(&yrow[k]) : __ldg(&yrow[k]) * __ldg(&wk[k])) * scale;
                const float cy0 = c * (1.f - t.ay), cy1 = c * t.ay;
                int* q = acc + lj * AW + li;
                atomicAdd(q, __float2int_rn(cy0 * (1.f - t.ax)));
                atomicAdd(q + 1, __float2int_rn(cy0 * t.ax));
                atomicAdd(q + AW, __float2int_rn(cy1 * (1.f - t.ax)));
                atomicAdd(q + AW + 1, __float2int_rn(cy1 * t.ax));
            }
        }
    }
    __syncthreads();
    // work items of one tile share its scale, so their fixed-point partial sums add
    // exactly (and in any order) with integer atomics
    for (int c = tid; c < WTILE * WTILE; c += ATHREADS) {
        const int lx = c % WTILE, ly = c / WTILE;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= N || gy >= N) continue;
        const int v = acc[(ly + 1) * AW + lx + 1];
        if (v) atomicAdd(&a.acc_out[(size_t)gy * N + gx], v);
    }
}

template <bool PREMUL>
__global__ void __launch_bounds__(ATHREADS, ADJ_MIN_BLOCKS) k_adjoint_tiles(AdjArgs a) {
    if (a.stop && *(volatile const int*)a.stop) return;
    adjoint_item<PREMUL>(a, blockIdx.x);
}

template <bool PREMUL>
__global__ void __launch_bounds__(ATHREADS, ADJ_MIN_BLOCKS) k_adjoint_tiles_b(const AdjArgs* __restrict__ args,
                                                            const int2* __restrict__ map) {
    const int2 pm = map[blockIdx.x];
    const AdjArgs& a = args[pm.x];   // (a shared copy would be reloaded after every shared atomic)
    if (a.stop && *(volatile const int*)a.stop) return;
    adjoint_item<PREMUL>(a, pm.y);
}

// out = the fixed-point K^T image in floating point
__global__ void k_kt_to_float(KtView kt, int N, float* __restrict__ out) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= N || gy >= N) return;
    out[(size_t)gy * N + gx] = kt.at(gx, gy, N);
}

// max of K^T 1 over each K^T tile, with headroom for the FP32 rounding of the terms
__global__ void k_tile_kmax(const float* __restrict__ kcol, int N, int tiles_x, float* __restrict__ tile_kmax) {
    const int t = blockIdx.x;
    const int x0 = (t % tiles_x) * ATILE, y0 = (t / tiles_x) * ATILE;
    float m = 0.f;
    for (int c = threadIdx.x; c < ATILE * ATILE; c += blockDim.x) {
        const int gx = x0 + c % ATILE, gy = y0 + c / ATILE;
        if (gx < N && gy < N) m = fmaxf(m, kcol[(size_t)gy * N + gx]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
        tile_kmax[t] = m * 1.0001f;
    }
}

// Row sums K 1 (FP64 accumulation) and column sums K^T 1 (FP64 atomics) of the
// nonnegative matrix K; only on-grid taps count.
__global__ void __launch_bounds__(128) k_precond_sums(GeomView g, float* __restrict__ krow,
                                                     double* __restrict__ kcol64) {
    const int d = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < g.n_t;
    const int2 w = __ldg(&g.win[d * g.n_kgrp + min(k / KGRP, g.n_kgrp - 1)]);
    const float2 det = __ldg(&g.det[d]);
    const float r = valid ? __ldg(&g.rk[k]) : 0.f;
    const double wk = valid ? (double)__ldg(&g.wk[k]) : 0.0;
    const int N = g.n;
    double acc = 0.0;
    int m = w.x;
    for (int j = 0; j < w.y; ++j) {
        const float2 cs = __ldg(&g.cs[m]);
        m = (m + 1 == g.quad_m) ? 0 : m + 1;
        Taps t;
        if (point_taps(g, det, r, cs, t) && valid) {
            const double ax = t.ax, ay = t.ay;
            const double wt[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};
            const int di[4] = {0, 1, 0, 1}, dj[4] = {0, 0, 1, 1};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = t.i0 + di[c], jj = t.j0 + dj[c];
                if (i >= 0 && i < N && jj >= 0 && jj < N) {
                    acc += wt[c];
                    atomicAdd(&kcol64[jj * N + i], wk * wt[c]);
                }
            }
        }
    }
    if (valid) krow[(size_t)d * g.n_t + k] = (float)(acc * wk);
}

__global__ void k_double_to_float(const double* __restrict__ a, float* __restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

static dim3 row_grid(const pat_geometry* g) {
    return dim3(ceil_div(g->desc.n_t, FWD_KW * KGRP), ceil_div(g->desc.n_det, FWD_DW));
}

int forward_row_blocks(const pat_geometry* g) {
    dim3 gr = row_grid(g);
    return gr.x * gr.y;
}

std::vector<float> forward_block_costs(const pat_geometry_desc& d, const std::vector<int2>& win) {
    const int D = d.n_det, n_kgrp = (d.n_t + KGRP - 1) / KGRP;
    const int nkb = ceil_div(d.n_t, FWD_KW * KGRP), ndb = ceil_div(D, FWD_DW);
    std::vector<float> cost((size_t)nkb * ndb, 0.f);
    for (int db = 0; db < ndb; ++db)
        for (int kb = 0; kb < nkb; ++kb) {
            float c = 0.f;
            for (int w = 0; w < ROW_WARPS; ++w) {   // the warp -> (detector, radii group) map of row_lane
                const int det = db * FWD_DW + w / FWD_KW, kg = kb * FWD_KW + w % FWD_KW;
                if (det < D && kg < n_kgrp) c += (float)win[(size_t)det * n_kgrp + kg].y;
            }
            cost[(size_t)db * nkb + kb] = c;   // local block index kb + nkb * db
        }
    return cost;
}


int launch_forward(const pat_geometry* g, const float* u, bool padded, float* y, cudaStream_t st) {
    (void)padded;
    k_forward<<<row_grid(g), ROW_THREADS, 0, st>>>(g->view, u, y);
    PAT_LAUNCH_CHECK("k_forward");
    return PAT_OK;
}

FwdProxArgs make_fwd_prox_args(const pat_geometry* g, const float4* ubar_quad, float* q, const float* f,
                               const float* sig_q, float sig_scalar, const float* step_mul, float* qw,
                               unsigned* qmax_bits, const int* stop) {
    FwdProxArgs a;
    a.g = g->view;
    a.ubar_quad = ubar_quad;
    a.q = q;
    a.f = f;
    a.sig_q = sig_q;
    a.sig_scalar = sig_scalar;
    a.step_mul = step_mul;
    a.qw = qw;
    a.qmax_bits = qmax_bits;
    a.stop = stop;
    return a;
}

FwdGapArgs make_fwd_gap_args(const pat_geometry* g, const float* u, const float4* u_quad, const float* q,
                             const float* f, double* partials, const int* stop) {
    FwdGapArgs a;
    a.g = g->view;
    a.u = u;
    a.u_quad = u_quad;
    a.q = q;
    a.f = f;
    a.partials = partials;
    a.stop = stop;
    return a;
}

int launch_forward_prox_b(const FwdProxArgs* args, const int2* map, int nblocks, cudaStream_t st) {
    if (nblocks <= 0) return PAT_OK;
    prof_mark(PAT_PHASE_FORWARD_PROX, st, true);
    k_forward_prox_b<<<nblocks, ROW_THREADS, 0, st>>>(args, map);
    PAT_LAUNCH_CHECK("k_forward_prox_b");
    prof_mark(PAT_PHASE_FORWARD_PROX, st, false);
    return PAT_OK;
}

int launch_forward_gap_b(const FwdGapArgs* args, const int2* map, int nblocks, cudaStream_t st) {
    if (nblocks <= 0) return PAT_OK;
    k_forward_gap_b<<<nblocks, ROW_THREADS, 0, st>>>(args, map);
    PAT_LAUNCH_CHECK("k_forward_gap_b");
    return PAT_OK;
}

int launch_absmax(const float* y, long long n, unsigned* out, cudaStream_t st) {
    k_absmax<<<std::min(4 * sm_count(), ceil_div(n, 256)), 256, 0, st>>>(y, n, out);
    PAT_LAUNCH_CHECK("k_absmax");
    return PAT_OK;
}

KtView kt_view(const pat_geometry* g, const int* acc, const unsigned* ymax_bits) {
    KtView v;
    v.acc = acc;
    v.ymax_bits = ymax_bits;
    v.tile_kmax = g->pc.tile_kmax;
    v.tiles_x = g->adj_tiles_x;
    return v;
}

AdjArgs make_adj_args(const pat_geometry* g, const float* y, const float* premul, const unsigned* ymax_bits, int* acc,
                      const int* stop) {
    AdjArgs a;
    a.g = g->view;
    a.y = premul ? premul : y;
    a.premul = premul ? 1 : 0;
    a.ymax_bits = ymax_bits;
    a.tile_kmax = g->pc.tile_kmax;
    a.rays = g->adj_rays;
    a.items = g->adj_item;
    a.acc_out = acc;
    a.tiles_x = g->adj_tiles_x;
    a.wtiles_x = g->adj_wtiles_x;
    a.stop = stop;
    return a;
}

int adjoint_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adjoint_tiles_b<true>, ATHREADS, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 4;
    }
    return n;
}

int launch_adjoint_b(const AdjArgs* args, const int2* map, int nblocks, bool premul, cudaStream_t st) {
    if (nblocks <= 0) return PAT_OK;
    prof_mark(PAT_PHASE_ADJOINT, st, true);
    if (premul)
        k_adjoint_tiles_b<true><<<nblocks, ATHREADS, 0, st>>>(args, map);
    else
        k_adjoint_tiles_b<false><<<nblocks, ATHREADS, 0, st>>>(args, map);
    PAT_LAUNCH_CHECK("k_adjoint_tiles_b");
    prof_mark(PAT_PHASE_ADJOINT, st, false);
    return PAT_OK;
}

static int launch_adjoint_fixed(const pat_geometry* g, const float* y, const float* premul,
                                const unsigned* ymax_bits, int* acc, const int* stop, cudaStream_t st) {
    const AdjArgs a = make_adj_args(g, y, premul, ymax_bits, acc, stop);
    if (a.premul)
        k_adjoint_tiles<true><<<g->adj_items, ATHREADS, 0, st>>>(a);
    else
        k_adjoint_tiles<false><<<g->adj_items, ATHREADS, 0, st>>>(a);
    PAT_LAUNCH_CHECK("k_adjoint_tiles");
    return PAT_OK;
}

// K^T y through caller-provided scratch: the max word at ymax_bits and the fixed-point
// image at acc (N*N int32), both already zero; no allocation and no profiling events.
int launch_adjoint_into(const pat_geometry* g, const float* y, unsigned* ymax_bits, int* acc, float* out,
                        cudaStream_t st) {
    const int N = g->desc.n;
    const long long S = (long long)g->desc.n_det * g->desc.n_t;
    k_absmax<<<std::min(4 * sm_count(), ceil_div(S, 256)), 256, 0, st>>>(y, S, ymax_bits);
    PAT_LAUNCH_CHECK("k_absmax");
    const AdjArgs a = make_adj_args(g, y, nullptr, ymax_bits, acc, nullptr);
    k_adjoint_tiles<false><<<g->adj_items, ATHREADS, 0, st>>>(a);
    PAT_LAUNCH_CHECK("k_adjoint_tiles");
    dim3 blk(32, 8), grd(ceil_div(N, 32), ceil_div(N, 8));
    k_kt_to_float<<<grd, blk, 0, st>>>(kt_view(g, acc, ymax_bits), N, out);
    PAT_LAUNCH_CHECK("k_kt_to_float");
    return PAT_OK;
}

int launch_adjoint(const pat_geometry* g, const float* y, float* out, cudaStream_t st) {
    int rc = ensure_precond(g, st);
    if (rc) return rc;
    const int N = g->desc.n;
    const size_t S = (size_t)g->desc.n_det * g->desc.n_t;
    char* scratch = nullptr;
    const size_t bytes = 256 + (size_t)N * N * sizeof(int);
    PAT_CUDA(cudaMallocAsync((void**)&scratch, bytes, st));
    unsigned* ymax = (unsigned*)scratch;
    int* acc = (int*)(scratch + 256);
    rc = cudaMemsetAsync(scratch, 0, bytes, st) == cudaSuccess ? PAT_OK : PAT_ERR_CUDA;
    if (!rc) {
        rc = launch_absmax(y, (long long)S, ymax, st);
        if (!rc) rc = launch_adjoint_fixed(g, y, nullptr, ymax, acc, nullptr, st);
    }
    if (!rc) {
        dim3 blk(32, 8), grd(ceil_div(N, 32), ceil_div(N, 8));
        k_kt_to_float<<<grd, blk, 0, st>>>(kt_view(g, acc, ymax), N, out);
        count_launch();
        rc = cudaGetLastError() == cudaSuccess ? PAT_OK : PAT_ERR_CUDA;
    }
    cudaFreeAsync(scratch, st);
    if (rc == PAT_ERR_CUDA) set_error("launch_adjoint: kernel launch failed");
    return rc;
}

int ensure_precond(const pat_geometry* gc, cudaStream_t st) {
    pat_geometry* g = const_cast<pat_geometry*>(gc);
    std::lock_guard<std::mutex> lock(g->mtx);
    if (g->pc.ready) return PAT_OK;
    const int N = g->desc.n;
    const size_t S = (size_t)g->desc.n_det * g->desc.n_t;
    if (!g->pc.krow) PAT_CUDA(cudaMalloc(&g->pc.krow, S * sizeof(float)));
    if (!g->pc.kcol) PAT_CUDA(cudaMalloc(&g->pc.kcol, (size_t)N * N * sizeof(float)));
    double* tmp = nullptr;
    PAT_CUDA(cudaMallocAsync(&tmp, (size_t)N * N * sizeof(double), st));
    PAT_CUDA(cudaMemsetAsync(tmp, 0, (size_t)N * N * sizeof(double), st));
    k_precond_sums<<<dim3(ceil_div(g->desc.n_t, 128), g->desc.n_det), 128, 0, st>>>(g->view, g->pc.krow, tmp);
    PAT_LAUNCH_CHECK("k_precond_sums");
    k_double_to_float<<<ceil_div((long long)N * N, 256), 256, 0, st>>>(tmp, g->pc.kcol, N * N);
    PAT_LAUNCH_CHECK("k_double_to_float");
    if (!g->pc.tile_kmax) PAT_CUDA(cudaMalloc(&g->pc.tile_kmax, (size_t)g->adj_tiles * sizeof(float)));
    k_tile_kmax<<<g->adj_tiles, 256, 0, st>>>(g->pc.kcol, N, g->adj_tiles_x, g->pc.tile_kmax);
    PAT_LAUNCH_CHECK("k_tile_kmax");
    PAT_CUDA(cudaFreeAsync(tmp, st));
    PAT_CUDA(cudaStreamSynchronize(st));
    g->pc.ready = true;
    return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" int pat_forward(const pat_geometry* g, const float* u_dev, float* y_dev, void* stream) {
    if (!g || !u_dev || !y_dev) return fail(PAT_ERR_INVALID_ARG, "pat_forward: NULL argument");
    return launch_forward(g, u_dev, false, y_dev, (cudaStream_t)stream);
}

extern "C" int pat_adjoint(const pat_geometry* g, const float* y_dev, float* u_dev, void* stream) {
    if (!g || !u_dev || !y_dev) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint: NULL argument");
    return launch_adjoint(g, y_dev, u_dev, (cudaStream_t)stream);
}
