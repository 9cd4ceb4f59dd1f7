// Exact transpose K^T of the circular-mean projector (Sec. 3.3.1, Sec. 4.2 eq. (K_def)) by
// pixel tiles with fixed-point accumulation, and the K^T entry points.
#include <algorithm>

#include "pat_internal.cuh"

namespace pat {

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
    const AdjGeom& g = a.g;
    const int N = g.n, T = g.n_t;
    const AdjItem* ip = a.items + item_index;
    const int tile = __ldg(&ip->tile), ray0 = __ldg(&ip->ray0), nray = __ldg(&ip->nray);
    const int c0 = __ldg(&ip->c0), c1 = __ldg(&ip->c1);
    const int x0 = (tile % a.wtiles_x) * WTILE, y0 = (tile / a.wtiles_x) * WTILE;
    const int tid = threadIdx.x;
    constexpr int AW = WTILE + 2;
    __shared__ int acc[AW * AW];
    __shared__ int4 s_ray[ARAYS + 1];   // {detector, angle, first k, prefix}
    __shared__ float4 s_geo[ARAYS];     // {detector x, y, cos / hx, sin / hy} of each segment
    for (int c = tid; c < AW * AW; c += ATHREADS) acc[c] = 0;
    for (int i = tid; i <= nray; i += ATHREADS) {
        s_ray[i] = __ldg(&a.rays[ray0 + i]);
        if (i < nray) s_geo[i] = __ldg(&a.ray_geo[ray0 + i]);
    }
    // the scale of the ATILE tile that holds this work tile
    const float bound = __uint_as_float(*a.ymax_bits) * __ldg(&a.tile_kmax[(y0 / ATILE) * a.tiles_x + x0 / ATILE]);
    const float scale = 1073741824.0f / bound;  // 2^30 / bound
    const float dr_f = g.dr_f, rh_f = g.rh_f;
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
            float4 geo = s_geo[j];
            float2 det = make_float2(geo.x, geo.y), cs = make_float2(geo.z, geo.w);
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
                    geo = s_geo[j];
                    det = make_float2(geo.x, geo.y);
                    cs = make_float2(geo.z, geo.w);
                    yrow = y + (size_t)ray.x * T;
                    k = ray.z;
                }
                Taps t;
                point_coords(g, det, radius(k, dr_f, rh_f), cs, t);   // = rk[k], bit for bit
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
    const GeomView& v = g->view;
    a.g = AdjGeom{v.n, v.n_t, v.det, v.cs, v.rk, v.wk, v.dr_f, v.rh_f};
    a.y = premul ? premul : y;
    a.premul = premul ? 1 : 0;
    a.ymax_bits = ymax_bits;
    a.tile_kmax = g->pc.tile_kmax;
    a.rays = g->adj_rays;
    a.ray_geo = g->adj_ray_geo;
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
    const int arc = launch_absmax(y, S, ymax_bits, st);
    if (arc) return arc;
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

}  // namespace pat

using namespace pat;

extern "C" int pat_adjoint(const pat_geometry* g, const float* y_dev, float* u_dev, void* stream) {
    if (!g || !u_dev || !y_dev) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint: NULL argument");
    return launch_adjoint(g, y_dev, u_dev, (cudaStream_t)stream);
}
