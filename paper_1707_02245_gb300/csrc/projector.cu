// Matrix-free circular-mean projector K (Sec. 3.3.1, Sec. 4.2 eq. (K_def)) with the fused
// data-row epilogues of the PDHG iteration, and the FP64 K sums of the preconditioners.
// Its exact transpose K^T is in adjoint.cu.
//
// K: every point of circle (d, k) is interpolated bilinearly between pixel centres.  The
// image is cut into S horizontal slabs, and a thread-block cluster of S CTAs holds the
// whole image: CTA s copies slab s (with a zero border and one extra row) into its shared
// memory and evaluates, for the cluster's row groups (8 radii of one detector), the
// points whose taps lie in its slab, so each of a point's four taps is a shared-memory
// load.  A warp holds the 8 radii of a row group times 4 angular phases, so at every step
// its 32 points form a 4-angle x 8-radius patch of the polar grid.  After a cluster
// barrier the S partial sums of a row are read through distributed shared memory and
// added in slab order, so the result does not depend on scheduling.  Images too large
// for the slabs of one cluster take the same units with taps from global memory.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "pat_internal.cuh"
#include "reduce.cuh"

namespace pat {

// Bilinear taps of a point from the plain N*N image in global memory, zero off the grid.
__device__ __forceinline__ float fetch4_global(const float* __restrict__ u, int N, const Taps& t, float& v10,
                                               float& v01, float& v11) {
    const bool x0 = t.i0 >= 0, x1 = t.i0 + 1 < N, y0 = t.j0 >= 0, y1 = t.j0 + 1 < N;
    const float* p = u + t.j0 * N + t.i0;
    v10 = (x1 && y0) ? __ldg(p + 1) : 0.f;
    v01 = (x0 && y1) ? __ldg(p + N) : 0.f;
    v11 = (x1 && y1) ? __ldg(p + N + 1) : 0.f;
    return (x0 && y0) ? __ldg(p) : 0.f;
}

// Lane mapping of a K unit: a warp holds the KGRP = 8 radii of one row group times NPH = 4
// angular phases, lane = ph * 8 + kl.  Phase ph walks a window at m_first + ph,
// m_first + ph + 4, ...  so at every step the warp evaluates a 4 (angles) x 8 (radii)
// patch of the polar grid, a compact patch of pixels.
constexpr int NPH = 4;
#ifndef PAT_FWD_PTS
#define PAT_FWD_PTS 2
#endif
constexpr int FWD_PTS = PAT_FWD_PTS;   // points per trip of the inner loop (independent sums)

// Sum over the four phases (lanes kl, kl+8, kl+16, kl+24); valid in every lane.
__device__ __forceinline__ float phase_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// Shared-memory loads by 32-bit shared address.
__device__ __forceinline__ float lds(unsigned a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds2(unsigned a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// 16-byte asynchronous copy global -> shared (no register staging), and its completion.
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Partial integral of the bilinear image over circle (d, k) for angular phase ph over the
// unit's two windows (each m_first | count << 16), counting only the points whose upper
// tap row j0 lies in [jlo, jlo + reff) and whose left tap column i0 lies in [-1, N-1].
//  SMEM: rows jlo .. jlo + reff of the zero-bordered image are staged in shared memory at
//  byte address img_s (column i at byte 4 (4 + i) of a row of W floats, with columns N and
//  N + 1 of rows 0 and 1 zero), and cs_s holds the angle table twice over, so m never
//  wraps.  The body has no branch: a point outside the slab or the grid reads the zero
//  cell at columns N, N + 1 of rows 0, 1.  FWD_PTS points per trip, with separate sums.
//  Otherwise: taps and angles come from global memory.
template <bool SMEM>
__device__ __forceinline__ float unit_partial(const GeomView& g, unsigned cs_s, const float* __restrict__ img,
                                              unsigned img_s, int jlo, int reff, unsigned w0, unsigned w1,
                                              float2 det, float r, bool valid, int ph) {
    const int N = g.n, M = g.quad_m, W = g.slab_stride;
    const int c0 = (int)(w0 >> 16), tot = c0 + (int)(w1 >> 16);
    const int m0 = (int)(w0 & 0xffffu), off1 = (int)(w1 & 0xffffu) - c0;   // m = j + (j < c0 ? m0 : off1)
    float acc = 0.f;
    if (SMEM) {
        const unsigned W4 = 4u * (unsigned)W;
        const unsigned base = img_s + 12u;                               // column i at base + 4 (i + 1)
        const unsigned zero = base + 4u * (unsigned)(N + 1);            // columns N, N + 1 of rows 0, 1
        const float2 rr = make_float2(r, r);
        const float2 mone = make_float2(-1.f, -1.f);
        const float2 magic = make_float2(FLOOR_MAGIC, FLOOR_MAGIC), nmagic = make_float2(-FLOOR_MAGIC, -FLOOR_MAGIC);
        const int lbias = FLOOR_MAGIC_BITS - 1;     // li = floor(fx) + 1
        const int jbias = FLOOR_MAGIC_BITS + jlo;   // lj = floor(fy) - jlo
        // FWD_PTS points per trip, each with its own partial sum (independent chains).  The
        // two windows run one after the other; in each, the lane's points are the window's
        // angles ph, ph + NPH, ... and their table entries are read at fixed offsets from
        // one address per trip.  Rows k >= T are evaluated like the others (their radius
        // is that of k = 0) and dropped at the end.
        float part[FWD_PTS];
#pragma unroll
        for (int e = 0; e < FWD_PTS; ++e) part[e] = 0.f;
        auto window = [&](int mstart, int cnt) {
            unsigned csp = cs_s + 8u * (unsigned)(mstart + ph);
            for (int j = ph; j < cnt; j += FWD_PTS * NPH, csp += 8u * FWD_PTS * NPH) {
#pragma unroll
                for (int e = 0; e < FWD_PTS; ++e) {
                    const bool vj = e == 0 || j + e * NPH < cnt;
                    const float2 cs = lds2(vj ? csp + 8u * NPH * e : csp);
                    // position and taps; the FP32 arithmetic of the transpose (fx = fmaf(r, cs.x, det.x))
                    const float2 fp = __ffma2_rn(rr, cs, det);
                    // exact floor (see point_coords): tp = floor(fp) + 1.5 * 2^23
                    const float2 tp = __fadd2_rd(fp, magic);
                    const int li = __float_as_int(tp.x) - lbias, lj = __float_as_int(tp.y) - jbias;
                    const bool in = ((unsigned)lj < (unsigned)reff) & ((unsigned)li <= (unsigned)N) & vj;
                    const unsigned ad = in ? base + (unsigned)lj * W4 + 4u * (unsigned)li : zero;   // li = i0 + 1
                    const float2 lo = make_float2(lds(ad), lds(ad + W4)), hi = make_float2(lds(ad + 4u), lds(ad + W4 + 4u));
                    // (ax, ay) = fp - floor(fp): floor(fp) = tp - C exactly, and the difference is exact
                    const float2 fr = __ffma2_rn(__fadd2_rn(tp, nmagic), mone, fp);
                    // rows j0 and j0 + 1 interpolated in x, then in y
                    const float2 pr = __ffma2_rn(make_float2(fr.x, fr.x), __ffma2_rn(lo, mone, hi), lo);
                    part[e] += fmaf(fr.y, pr.y - pr.x, pr.x);
                }
            }
        };
        window(m0, c0);
        window((int)(w1 & 0xffffu), (int)(w1 >> 16));
#pragma unroll
        for (int e = 1; e < FWD_PTS; ++e) part[0] += part[e];
        acc = valid ? part[0] : 0.f;
    } else {
        for (int j = ph; j < tot; j += NPH) {
            const int mm = j + (j < c0 ? m0 : off1);
            const int m = mm >= M ? mm - M : mm;
            Taps t;
            point_coords(g, det, r, __ldg(&g.cs[m]), t);
            if ((unsigned)(t.j0 + 1) <= (unsigned)N && (unsigned)(t.i0 + 1) <= (unsigned)N && valid) {
                float v10, v01, v11;
                const float v00 = fetch4_global(img, N, t, v10, v01, v11);
                const float p = fmaf(t.ax, v10 - v00, v00);
                const float q = fmaf(t.ax, v11 - v01, v01);
                acc += fmaf(t.ay, q - p, p);
            }
        }
    }
    return acc;
}

// Issues the copy of image rows jlo .. jlo + nrow - 1 into the slab at s_img (row t at
// float t W, column i at float t W + 4 + i): cp.async for rows inside the image when N is
// a multiple of 4 and the image 16-byte aligned, plain loads otherwise; rows outside the
// image and the columns -1 and N are zero.  Completed by cp_async_wait_all() and a barrier.
template <int NT>
__device__ __forceinline__ void stage_slab(const float* __restrict__ img, int N, int W, int jlo, int nrow,
                                           float* s_img) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (N & 3) == 0 && ((reinterpret_cast<size_t>(img) & 15) == 0);
    const unsigned base = smem_addr(s_img);
    for (int t = warp; t < nrow; t += NT / 32) {
        const int j = jlo + t;
        float* row = s_img + t * W;
        const bool in = j >= 0 && j < N;
        if (vec && in) {
            const float* src = img + (size_t)j * N;
            for (int c = 4 * lane; c < N; c += 128) cp_async16(base + 4u * (unsigned)(t * W + 4 + c), src + c);
        } else {
            for (int c = lane; c < N; c += 32) row[4 + c] = in ? __ldg(img + (size_t)j * N + c) : 0.f;
        }
        if (lane == 0) {
            row[3] = 0.f;
            row[4 + N] = 0.f;
            if (t < 2) row[5 + N] = 0.f;   // with column N: the zero cell of out-of-slab points
        }
    }
}

// Shared-memory layout of a K CTA (byte offsets; every part 16-byte aligned):
//   slab image (R + 1) * W floats | the round's units (at most FWD_ROUND) | cs twice over
//   (2M float2) | det (D float2) | the round's accumulators (FWD_ROUND * KGRP floats)
struct FwdSmem {
    int slab, units, cs, det, acc, total;
};
__host__ __device__ __forceinline__ int align16(int x) { return (x + 15) & ~15; }
__host__ __device__ __forceinline__ FwdSmem fwd_smem_layout(int rows, int stride, int M, int D, bool staged) {
    FwdSmem l;
    l.slab = 0;
    l.units = align16(rows > 0 ? (rows + 1) * stride * 4 : 0);
    l.cs = l.units + FWD_ROUND * 16;
    l.det = l.cs + (staged ? align16(2 * M * 8) : 0);   // the angle table twice over
    l.acc = l.det + (staged ? align16(D * 8) : 0);
    l.total = l.acc + FWD_ROUND * KGRP * 4;
    return l;
}

// cluster helpers: rank in the cluster, barrier over the cluster's CTAs (orders shared
// memory writes before the barrier with reads after it), and a load from the shared
// memory of CTA `rank` at the offset of the local address p
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float ld_cluster(const float* p, unsigned rank) {
    unsigned a = smem_addr(p), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}

// One round of a CTA: warps take the CTA's units of the round one at a time and store each
// unit's row sums in the accumulators of its row group (one unit per row group and CTA).
template <bool SMEM>
__device__ __forceinline__ void forward_units(const FwdArgs& a, int ub, int ue, unsigned char* smem,
                                              const FwdSmem& L, int jlo, int reff, int& s_next) {
    const GeomView& g = a.g;
    const int T = g.n_t;
    const int4* s_units = reinterpret_cast<const int4*>(smem + L.units);
    const float2* s_det = reinterpret_cast<const float2*>(smem + L.det);
    float* s_acc = reinterpret_cast<float*>(smem + L.acc);
    const unsigned img_s = smem_addr(smem + L.slab), cs_s = smem_addr(smem + L.cs);
    const float dr_f = g.dr_f, rh_f = g.rh_f;
    const int lane = threadIdx.x & 31, kl = lane & 7, ph = lane >> 3;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(&s_next, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= ue) break;
        const int4 un = s_units[u - ub];
        const int d = un.x;
        const int k = (un.w >> 16) * KGRP + kl;
        const bool valid = k < T;
        const float r = radius(valid ? k : 0, dr_f, rh_f);   // = rk[k], bit for bit
        const float2 det = SMEM ? s_det[d] : __ldg(&g.det[d]);
        const float acc = unit_partial<SMEM>(g, cs_s, a.img, img_s, jlo, reff, (unsigned)un.y, (unsigned)un.z, det, r,
                                             valid, ph);
        const float sum = phase_sum(acc);
        if (ph == 0) s_acc[(un.w & 0xffff) * KGRP + kl] = sum;
    }
}

// K (Sec. 3.3.1, eq. (K_def)) for the row groups of one cluster, then the epilogue on
// their rows.  The S partial sums of a row (one per slab) are added in rank (slab) order,
// so the result does not depend on scheduling.
template <int EPI, int NT>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : 2) k_forward_b(const FwdArgs* __restrict__ args,
                                                           const int2* __restrict__ map) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ FwdArgs sa;
    __shared__ int s_next;
    __shared__ unsigned s_qmax;
    const int2 pm = map[blockIdx.x];
    const FwdArgs& a = stage_args(args, pm.x, sa);
    // (every CTA of a cluster reads the same flag, so a stopped problem's clusters leave
    // together, before any cluster barrier)
    if (a.stop && *(volatile const int*)a.stop) return;
    const GeomView& g = a.g;
    const int N = g.n, T = g.n_t, S = g.n_slabs, M = g.quad_m, D = g.n_det;
    const unsigned rank = S > 1 ? cluster_rank() : 0u;
    const int4 cta = __ldg(&g.ctas[pm.y]);
    const int rg0 = cta.x, n_rg = cta.y;
    const int* roff = g.roff + cta.z;
    const bool smem_img = g.slab_rows > 0;
    const FwdSmem L = fwd_smem_layout(g.slab_rows, g.slab_stride, M, D, smem_img);
    float* s_acc = reinterpret_cast<float*>(smem + L.acc);
    int4* s_units = reinterpret_cast<int4*>(smem + L.units);
    const int jlo = smem_img ? (int)rank * g.slab_rows - 1 : -1;
    const int reff = smem_img ? min(g.slab_rows, N - jlo) : N + 1;
    if (smem_img) {
        float2* s_cs = reinterpret_cast<float2*>(smem + L.cs);
        float2* s_det = reinterpret_cast<float2*>(smem + L.det);
        for (int i = threadIdx.x; i < 2 * M; i += NT) s_cs[i] = __ldg(&g.cs[i < M ? i : i - M]);
        for (int i = threadIdx.x; i < D; i += NT) s_det[i] = __ldg(&g.det[i]);
        stage_slab<NT>(a.img, N, g.slab_stride, jlo, reff + 1, reinterpret_cast<float*>(smem + L.slab));
    }
    if (threadIdx.x == 0) s_qmax = 0u;
    const int lane = threadIdx.x & 31;
    const float smul = (EPI == FWD_PROX && a.step_mul) ? __ldg(a.step_mul + 1) : 1.f;
    unsigned qbits = 0u;
    float t[GAP_DATA_TERMS] = {0.f, 0.f, 0.f, 0.f};
    const int n_rounds = (n_rg + FWD_ROUND - 1) / FWD_ROUND;
    for (int rd = 0; rd < n_rounds; ++rd) {
        const int ub = __ldg(&roff[rd]), ue = __ldg(&roff[rd + 1]);
        const int nr = min(FWD_ROUND, n_rg - rd * FWD_ROUND);
        for (int i = threadIdx.x; i < ue - ub; i += NT) s_units[i] = __ldg(&g.units[ub + i]);
        for (int i = threadIdx.x; i < nr * KGRP; i += NT) s_acc[i] = 0.f;
        if (threadIdx.x == 0) s_next = ub;
        if (smem_img && rd == 0) cp_async_wait_all();
        __syncthreads();
        if (smem_img)
            forward_units<true>(a, ub, ue, smem, L, jlo, reff, s_next);
        else
            forward_units<false>(a, ub, ue, smem, L, jlo, reff, s_next);
        // all CTAs of the cluster have their partial sums of the round
        if (S > 1) cluster_sync(); else __syncthreads();
        // epilogue: the round's rows are split over the cluster's CTAs; row i of the round
        // is row (i % KGRP) of row group rgs[rg0 + rd * FWD_ROUND + i / KGRP]
        const int rows = nr * KGRP, per = (rows + S - 1) / S;
        const int i0 = (int)rank * per, i1 = min(rows, i0 + per);
        for (int i = i0 + threadIdx.x; i < i1; i += NT) {
            const int rg = __ldg(&g.rgs[rg0 + rd * FWD_ROUND + i / KGRP]);
            const int d = rg / g.n_kgrp;
            const int k = (rg - d * g.n_kgrp) * KGRP + (i & (KGRP - 1));
            if (k >= T) continue;
            float sum = 0.f;
            for (int r = 0; r < S; ++r) sum += (S > 1) ? ld_cluster(&s_acc[i], (unsigned)r) : s_acc[i];
            const size_t row = (size_t)d * T + k;
            const float wk = __ldg(&g.wk[k]);
            if (EPI == FWD_Y) {
                a.y[row] = sum * wk;
            } else if (EPI == FWD_PROX) {
                // q <- prox_{sigma F1*}(q + sigma K ubar) = (q + sigma (K ubar - f)) / (1 + sigma)  (Sec. 3.2)
                const float ku = sum * wk;
                const float sg = (a.sig_q ? a.sig_q[row] : a.sig_scalar) * smul;
                const float qn = (a.q[row] + sg * (ku - a.f[row])) / (1.f + sg);
                a.q[row] = qn;
                a.qw[row] = qn * wk;
                qbits = max(qbits, __float_as_uint(fabsf(qn)));  // a NaN's bits exceed every finite value's
            } else {
                // per-row terms in FP32; the CTA's sums as FP32 pairs per warp, FP64 across warps
                const float ku = sum * wk;
                const float res = ku - a.f[row];
                const float qi = a.q[row];
                t[0] += res * res;
                t[1] += qi * qi;
                t[2] += qi * a.f[row];
                t[3] += fabsf(qi - res);   // dual residual of the data term: q - dF1(Ku)
            }
        }
        // the accumulators and units are reused by the next round, and no CTA may leave
        // while another still reads its accumulators
        if (S > 1) cluster_sync(); else __syncthreads();
    }
    if (EPI == FWD_PROX) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qbits = max(qbits, __shfl_xor_sync(0xffffffffu, qbits, o));
        if (lane == 0 && qbits) atomicMax(&s_qmax, qbits);
        __syncthreads();
        if (threadIdx.x == 0 && s_qmax) atomicMax(a.qmax_bits, s_qmax);
    }
    if (EPI == FWD_GAP) {
        double sum[GAP_DATA_TERMS];
        block_sum_pair<GAP_DATA_TERMS>(t, sum);
        if (threadIdx.x == 0)
            for (int c = 0; c < GAP_DATA_TERMS; ++c) a.partials[(size_t)GAP_DATA_TERMS * pm.y + c] = sum[c];
    }
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

FwdArgs make_fwd_args(const pat_geometry* g, const float* img) {
    FwdArgs a;
    memset(&a, 0, sizeof a);
    a.g = g->view;
    a.img = img;
    return a;
}

int forward_smem_bytes(int rows, int stride, int M, int D, bool staged) {
    return fwd_smem_layout(rows, stride, M, D, staged).total;
}

// K launches may use up to FWD_SMEM_ONE bytes of dynamic shared memory; the attribute is
// set once per kernel and device.
template <int NT>
static cudaError_t forward_attributes_nt() {
    const void* ks[3] = {(const void*)k_forward_b<FWD_Y, NT>, (const void*)k_forward_b<FWD_PROX, NT>,
                         (const void*)k_forward_b<FWD_GAP, NT>};
    for (const void* k : ks) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM_ONE);
        if (e != cudaSuccess) return e;
        // clusters of more than 8 CTAs (up to FWD_MAX_CLUSTER) where the device allows them
        if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
    }
    return cudaSuccess;
}

static int forward_attributes() {
    static std::mutex mtx;
    static bool done[64] = {};
    int dev = 0;
    PAT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mtx);
    if (dev >= 0 && dev < 64 && done[dev]) return PAT_OK;
    PAT_CUDA(forward_attributes_nt<FWD_THREADS>());
    PAT_CUDA(forward_attributes_nt<FWD_THREADS_WIDE>());
    if (dev >= 0 && dev < 64) done[dev] = true;
    return PAT_OK;
}

// Threads of a K CTA: a CTA whose shared memory leaves no room for a second one on its SM
// runs twice as many warps, so that the SM keeps the same number of warps in flight.
int forward_threads(int smem) { return smem > FWD_SMEM_TWO ? FWD_THREADS_WIDE : FWD_THREADS; }

static cudaLaunchConfig_t forward_config(int nblocks, int cluster, int smem, cudaStream_t st,
                                         cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)forward_threads(smem));
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int forward_clusters_per_gpu(int cluster, int smem) {
    int n = 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = forward_config(cluster, cluster, smem, nullptr, attr);
    const void* k = forward_threads(smem) == FWD_THREADS_WIDE ? (const void*)k_forward_b<FWD_PROX, FWD_THREADS_WIDE>
                                                              : (const void*)k_forward_b<FWD_PROX, FWD_THREADS>;
    if (forward_attributes() != PAT_OK || cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return n;   // 0: clusters of this shape cannot run on the device
}

template <int NT>
static cudaError_t launch_forward_nt(int epi, const cudaLaunchConfig_t& cfg, const FwdArgs* args, const int2* map) {
    if (epi == FWD_Y) return cudaLaunchKernelEx(&cfg, k_forward_b<FWD_Y, NT>, args, map);
    if (epi == FWD_PROX) return cudaLaunchKernelEx(&cfg, k_forward_b<FWD_PROX, NT>, args, map);
    return cudaLaunchKernelEx(&cfg, k_forward_b<FWD_GAP, NT>, args, map);
}

int launch_forward_b(int epi, const FwdArgs* args, const int2* map, int nblocks, int cluster, int smem,
                     cudaStream_t st) {
    if (nblocks <= 0) return PAT_OK;
    const int arc = forward_attributes();
    if (arc) return arc;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = forward_config(nblocks, cluster, smem, st, attr);
    if (epi == FWD_PROX) prof_mark(PAT_PHASE_FORWARD_PROX, st, true);
    const cudaError_t e = forward_threads(smem) == FWD_THREADS_WIDE ? launch_forward_nt<FWD_THREADS_WIDE>(epi, cfg, args, map)
                                                                    : launch_forward_nt<FWD_THREADS>(epi, cfg, args, map);
    count_launch();
    if (e != cudaSuccess) return cuda_fail(e, "k_forward_b");
    if (epi == FWD_PROX) prof_mark(PAT_PHASE_FORWARD_PROX, st, false);
    return PAT_OK;
}

int launch_forward(const pat_geometry* g, const float* u, float* y, cudaStream_t st) {
    const int nc = g->fwd_n_ctas;
    const size_t map_off = (sizeof(FwdArgs) + 255) & ~(size_t)255;
    const size_t bytes = map_off + (size_t)nc * sizeof(int2);
    char* buf = nullptr;
    PAT_CUDA(cudaMallocAsync((void**)&buf, bytes, st));
    FwdArgs a = make_fwd_args(g, u);
    a.y = y;
    std::vector<int2> map(nc);
    for (int i = 0; i < nc; ++i) map[i] = make_int2(0, i);
    int rc = PAT_OK;
    cudaError_t e = cudaMemcpyAsync(buf, &a, sizeof a, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf + map_off, map.data(), (size_t)nc * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "launch_forward: arguments");
    // (copies from pageable host memory are staged before cudaMemcpyAsync returns, so the
    // host arguments may go out of scope)
    if (!rc)
        rc = launch_forward_b(FWD_Y, (const FwdArgs*)buf, (const int2*)(buf + map_off), nc, g->view.n_slabs,
                              g->fwd_smem, st);
    cudaFreeAsync(buf, st);
    return rc;
}

int launch_absmax(const float* y, long long n, unsigned* out, cudaStream_t st) {
    k_absmax<<<std::min(4 * sm_count(), ceil_div(n, 256)), 256, 0, st>>>(y, n, out);
    PAT_LAUNCH_CHECK("k_absmax");
    return PAT_OK;
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
    return launch_forward(g, u_dev, y_dev, (cudaStream_t)stream);
}

