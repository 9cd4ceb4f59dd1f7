// Internal declarations of the PDHG photoacoustic library (CUDA, sm_103a).
// Shared by the translation units of the library only; the public boundary is pat.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "pat.h"

namespace pat {

// ---------------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PAT_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return ::pat::cuda_fail(e_, #call);  \
    } while (0)

void count_launch();
int sm_count();   // SMs of the current device (sizes grid-stride launches)

// Every kernel launch of the library is followed by this check, which also counts it.
#define PAT_LAUNCH_CHECK(what)                                      \
    do {                                                            \
        ::pat::count_launch();                                      \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return ::pat::cuda_fail(e_, what);   \
    } while (0)

// Optional per-phase timing: marks record a CUDA event pair around a phase when the
// profiler is on; prof_collect() (after the stream has synchronised) adds the elapsed
// times to the process-wide sums.
bool prof_on();
void prof_mark(int phase, cudaStream_t st, bool begin);
void prof_collect();

// ---------------------------------------------------------------------------------
// device view of a geometry (passed by value to kernels)
// ---------------------------------------------------------------------------------
// Quadrature point m of circle (d, k) in continuous pixel coordinates (fp32):
//   fx = det[d].x + r[k] * cs[m].x   with det = ((x_d - xmin)/hx - 1/2, (y_d - ymin)/hy - 1/2)
//                                    and  cs = (cos(phi_m)/hx, sin(phi_m)/hy)   (from FP64)
// so pixel (i, j) has its centre at fx = i, fy = j.  Taps i0 = floor(fx), i0 + 1 with
// weights 1 - ax, ax (ax = fx - i0); same in y.
// K works on row groups: KGRP consecutive radii of one detector (row group rg = d *
// n_kgrp + k / KGRP).  The image is cut into S horizontal slabs of R rows of upper tap
// rows j0 (slab s holds the points with j0 in [s R - 1, (s + 1) R - 1)).  K runs as
// clusters of S CTAs: CTA rank s stages slab s in shared memory once, and the cluster owns
// a list of row groups, processed in rounds of at most FWD_ROUND row groups.  In a round,
// each CTA evaluates its slab's work units (one row group restricted to one slab: at most
// two circular angular windows) into its shared accumulators; after a cluster barrier the
// rows' S partial sums are added in rank order through distributed shared memory and the
// epilogue runs.  slab_rows = 0 marks the global-memory variant (S = 1, no staging) used
// when the image does not fit a cluster of at most FWD_MAX_CLUSTER CTAs.
struct GeomView {
    int n, n_det, n_t, quad_m;
    int n_kgrp;          // k groups of KGRP consecutive radii per detector
    const float2* det;   // D detector positions in continuous pixel coordinates
    const float2* cs;    // M (cos phi_m / hx, sin phi_m / hy)
    const float* rk;     // T radii, rk[k] = fmaf(k, dr_f, rh_f) (see radius())
    const float* wk;     // T arc weights 2 pi r_k / M
    const int2* win;     // D * n_kgrp angular windows {m_first, m_count} (circular)
    float dr_f, rh_f;    // FP32 radius step dr and first radius r0 + dr/2
    int n_slabs;         // S >= 1: slabs, and CTAs per cluster
    int slab_rows;       // R (0: global-memory variant)
    int slab_stride;     // shared-memory row stride in floats (W = 4 mod 8, >= N + 6)
    int smem_bytes;      // dynamic shared memory of a K CTA of this plan
    // units {detector, window 0, window 1, (k group << 16) | row group's index in its
    // round}; a window is m_first | count << 16.  A CTA's units are stored round by round.
    const int4* units;
    const int4* ctas;    // per K CTA (cluster-major, rank-minor): {first entry in rgs, row groups, first entry in roff, 0}
    const int* roff;     // per CTA: unit offsets of its rounds (rounds + 1 entries)
    const int* rgs;      // per cluster: its row groups in processing order
};

// Radius r_k = r0 + (k + 1/2) dr in FP32, as one correctly rounded fused multiply-add of
// FP32 constants; the host builds the radius table with the same expression (std::fmaf is
// correctly rounded too), so a kernel may evaluate it instead of loading rk[k].
__host__ __device__ __forceinline__ float radius(int k, float dr_f, float rh_f) {
    return fmaf((float)k, dr_f, rh_f);
}

constexpr int KGRP = 8;        // radii per angular-window group
constexpr int FWD_THREADS = 512;        // threads of a K CTA (two CTAs per SM)
constexpr int FWD_THREADS_WIDE = 1024;  // threads of a K CTA that holds its SM alone
constexpr int FWD_SMEM_TWO = 112 * 1024;         // dynamic shared memory of a K CTA, two per SM
constexpr int FWD_SMEM_ONE = 220 * 1024;         // ... one per SM
constexpr int FWD_MAX_CLUSTER = 16;              // largest (non-portable) cluster size
constexpr int FWD_ROUND = 256;                   // row groups of a cluster per round
constexpr int FWD_STAGE_MAX = 1024;              // slabs need the cs and det tables staged: M, D <= this
constexpr int MAX_QUAD_M = 8192;
constexpr int ATILE = 32;      // side of the pixel tiles that share one K^T fixed-point scale
constexpr int WTILE = 32;      // side of the pixel tiles one K^T work item accumulates
static_assert(ATILE % WTILE == 0, "work tiles nest in scale tiles");
constexpr int ARAYS = 1024;    // most ray segments one K^T work item holds
#ifndef PAT_ADJ_WAVES
#define PAT_ADJ_WAVES 1
#endif
constexpr int ADJ_WAVES = PAT_ADJ_WAVES;   // waves of resident CTAs the K^T work items fill

// One K^T work item: candidates [c0, c1) of work tile `tile`'s concatenated ray segments,
// which lie on the nray segments rays[ray0 .. ray0 + nray); rays[ray0 + nray] is the next
// segment of the tile or its sentinel, whose prefix ends the last segment.
struct AdjItem {
    int tile, ray0, nray, c0, c1, pad0, pad1, pad2;
};

struct PrecondCache {
    float* krow = nullptr;      // K 1 per data row (S), summed in FP64
    float* kcol = nullptr;      // K^T 1 per pixel (N*N), summed in FP64
    float* tile_kmax = nullptr; // max of K^T 1 over each K^T tile
    bool ready = false;
};

}  // namespace pat

struct pat_geometry {
    pat_geometry_desc desc;
    int device = 0;
    long long points_per_apply = 0;   // quadrature points inside the windows (evaluated)
    long long points_on_grid = 0;     // quadrature points whose taps touch the grid
    // device tables
    float2* det = nullptr;
    float2* cs = nullptr;
    float* rk = nullptr;
    float* wk = nullptr;
    int2* win = nullptr;
    int4* adj_rays = nullptr;         // K^T ray segments {detector, angle, first k, prefix}, per tile + sentinel
    float4* adj_ray_geo = nullptr;    // per segment {det.x, det.y, cs.x, cs.y} of the FP32 tables
    pat::AdjItem* adj_item = nullptr;  // K^T work items, one CTA each
    int adj_tiles_x = 0, adj_tiles = 0, adj_items = 0;   // scale tiles (ATILE) per row, in all; items
    int adj_wtiles_x = 0;              // work tiles (WTILE) per row
    long long adj_candidates = 0;     // candidate points of one K^T application
    std::vector<float> adj_item_cost;  // estimated cost per work item (host)
    int4* fwd_units = nullptr;         // K work units (see GeomView)
    int4* fwd_ctas = nullptr;          // K CTAs
    int* fwd_roff = nullptr;           // per CTA: unit offsets of its rounds
    int* fwd_rgs = nullptr;            // per cluster: its row groups
    int fwd_n_ctas = 0, fwd_smem = 0;  // K CTAs of one application (clusters x S); dynamic shared memory
    long long fwd_evaluated = 0;       // quadrature points inside the units' windows
    std::vector<float> fwd_cluster_cost; // points each K cluster's slowest CTA evaluates (host)
    std::vector<double> det_xy;        // detector positions (host copy, 2 per detector)
    std::vector<int2> win_host;        // angular windows over the grid (host copy)
    pat_shapes shapes{};               // launch shapes in use (see pat_geometry_set_shapes)
    int fwd_requested = PAT_FWD_AUTO;  // the K variant last asked for (shapes.forward: resolved)
    pat::GeomView view;
    // lazily computed preconditioner sums
    mutable std::mutex mtx;
    mutable pat::PrecondCache pc;
};

namespace pat {

// ---------------------------------------------------------------------------------
// shared device helpers
// ---------------------------------------------------------------------------------
struct Taps {
    int i0, j0;
    float ax, ay;
};

// Position of quadrature point (d, k, m) and its bilinear taps.  Returns false when no
// tap can touch the grid (i0 or j0 outside [-1, N-1]).
__device__ __forceinline__ bool point_taps(const GeomView& g, float2 det, float r, float2 cs,
                                           Taps& t) {
    const float fx = fmaf(r, cs.x, det.x);
    const float fy = fmaf(r, cs.y, det.y);
    const float flx = floorf(fx);
    const float fly = floorf(fy);
    t.ax = fx - flx;
    t.ay = fy - fly;
    // geometry creation bounds |fx|, |fy| by 2^22, so the conversions are exact
    t.i0 = (int)flx;
    t.j0 = (int)fly;
    return (unsigned)(t.i0 + 1) <= (unsigned)g.n && (unsigned)(t.j0 + 1) <= (unsigned)g.n;
}

// K^T y held as int32 fixed point: pixel p stores round((K^T y)(p) * S_t) with the
// per-tile scale S_t = 2^30 / (max|y| * max over tile t of K^T 1).
struct KtView {
    const int* acc;             // N*N
    const unsigned* ymax_bits;  // max |y| as float bits
    const float* tile_kmax;     // per tile
    int tiles_x;
    // the factor that turns tile (tx, ty)'s fixed-point sums into values: bound * 2^-30
    __device__ __forceinline__ float inv_scale(int tx, int ty) const {
        const float bound = __uint_as_float(*ymax_bits) * __ldg(&tile_kmax[ty * tiles_x + tx]);
        return bound > 0.f ? bound * 9.313225746154785e-10f : (bound == 0.f ? 0.f : bound);
    }
    __device__ __forceinline__ float at(int gx, int gy, int N) const {
        return (float)__ldg(&acc[(size_t)gy * N + gx]) * inv_scale(gx / ATILE, gy / ATILE);
    }
};

// Exact floor of x and its integer for |x| < 2^22, on the FMA and integer pipes (no
// conversion instructions): t = x + 1.5 * 2^23 rounded down lies in [2^23, 2^24), where the
// spacing of floats is 1, so t = floor(x) + 1.5 * 2^23 exactly; then floor(x) = t - 1.5 *
// 2^23 (exact) and its integer is the low bits of t.  Geometry creation bounds the
// continuous pixel coordinates of every quadrature point by 2^22.
constexpr float FLOOR_MAGIC = 12582912.0f;   // 1.5 * 2^23, bits 0x4B400000
constexpr int FLOOR_MAGIC_BITS = 0x4B400000;

// Taps of a point without the grid test (callers that test a tile window instead).  The
// floors are floorf (K's shared-memory loop takes the same floors by the exact round-down
// add above; here floorf measured faster: K^T 26.3 against 29.4 us at 256^2).
template <class G>
__device__ __forceinline__ void point_coords(const G& g, float2 det, float r, float2 cs, Taps& t) {
    const float fx = fmaf(r, cs.x, det.x);
    const float fy = fmaf(r, cs.y, det.y);
    const float flx = floorf(fx);
    const float fly = floorf(fy);
    t.ax = fx - flx;
    t.ay = fy - fly;
    t.i0 = (int)flx;
    t.j0 = (int)fly;
}

// Launch helpers
inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// p moved on by b bytes: problem k of a batch whose per-problem buffers lie a fixed byte
// stride apart reads its buffers at the first problem's pointers plus k times that stride
template <class T>
__host__ __device__ __forceinline__ T* at_bytes(T* p, long long b) {
    return (T*)((const char*)p + b);
}

// Copies problem p's argument struct into the block's shared copy (one word per thread)
// so that field reads are shared-memory broadcasts; ends with a block barrier.
template <class T>
__device__ __forceinline__ const T& stage_args(const T* __restrict__ args, int p, T& smem) {
    static_assert(sizeof(T) % 4 == 0, "argument structs are whole words");
    constexpr int W = (int)(sizeof(T) / 4);
    const int* src = reinterpret_cast<const int*>(args + p);
    int* dst = reinterpret_cast<int*>(&smem);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int i = tid; i < W; i += nt) dst[i] = src[i];
    __syncthreads();
    return smem;
}

// ---------------------------------------------------------------------------------
// per-problem kernel arguments of the batched launches: a launch covers several problems,
// block b of the launch works on problem map[b].x, local block map[b].y
// ---------------------------------------------------------------------------------
// K applied to an N*N image for every row group of one problem, with one of three
// epilogues on the finished rows: FWD_Y writes y = K img; FWD_PROX performs the data prox
// q <- (q + sigma (K ubar - f)) / (1 + sigma) and records q w_k and max |q| for the K^T
// that follows; FWD_GAP writes the per-row-group sums of the gap's data terms.
enum { FWD_Y = 0, FWD_PROX = 1, FWD_GAP = 2 };
constexpr int GAP_DATA_TERMS = 4;   // per-row-group sums of the data pass: |Ku-f|^2, |q|^2, <q,f>, |q-(Ku-f)|_1

struct FwdArgs {
    GeomView g;
    const float* img;      // N*N row-major image (ubar, or u for the gap)
    float* y;              // FWD_Y: D*T
    float* q;              // FWD_PROX, FWD_GAP
    const float* f;
    const float* sig_q;    // NULL: sig_scalar
    float sig_scalar;
    const float* step_mul; // {tau multiplier s, sigma multiplier 1/s} (device) or NULL
    float* qw;
    unsigned* qmax_bits;
    double* partials;      // FWD_GAP: one GAP_DATA_TERMS block of sums per K CTA
    const int* stop;
};

// The geometry fields K^T reads (a compact copy: each CTA reads its arguments from
// global memory, and the full view measured 3 us slower per launch at 256^2)
struct AdjGeom {
    int n, n_t;
    const float2* det;
    const float2* cs;
    const float* rk;
    const float* wk;
    float dr_f, rh_f;
};

struct AdjArgs {       // fixed-point K^T y, one work item per block
    AdjGeom g;
    const float* y;          // data rows, or data rows times the arc weights (premul)
    int premul;
    const unsigned* ymax_bits;
    const float* tile_kmax;
    const int4* rays;
    const float4* ray_geo;   // per segment: its detector and direction, from the FP32 tables
    const AdjItem* items;
    int* acc_out;            // N*N fixed-point image, added to with integer atomics
    int tiles_x;             // scale tiles per row
    int wtiles_x;            // work tiles per row
    const int* stop;
};

FwdArgs make_fwd_args(const pat_geometry* g, const float* img);
AdjArgs make_adj_args(const pat_geometry* g, const float* y, const float* premul, const unsigned* ymax_bits, int* acc,
                      const int* stop);
// batched launches over maps of (problem, local block); args are device arrays by problem
// K launch over a map of (problem, CTA) pairs: cluster-major, the S ranks of a cluster
// consecutive; every problem of one launch has the same S (cluster size).  smem: dynamic
// shared memory of the launch (the largest plan of its problems).
int launch_forward_b(int epi, const FwdArgs* args, const int2* map, int nblocks, int cluster, int smem,
                     cudaStream_t st);
int forward_smem_bytes(int rows, int stride, int M, int D, bool staged);
int forward_clusters_per_gpu(int cluster, int smem);   // K clusters the GPU holds at once
int forward_threads(int smem);                         // threads of a K CTA with this shared memory
int launch_adjoint_b(const AdjArgs* args, const int2* map, int nblocks, bool premul, cudaStream_t st);
// CTAs of the K^T kernel that one SM holds at once (sizes the work items)
int adjoint_blocks_per_sm();


// Host entry points implemented in projector.cu and used by pdhg.cu
// ---- the wavelet model (wavelet.cu) ----
struct WavPrimalArgs {   // u <- u - T (K^T q + W^T r) / s, ubar, and the next parity's reset
    int n;
    const float* scal;   // {alpha, theta}
    const float* tau_u;
    const float* step_mul;
    KtView kt;
    const float* wtr;
    float* u;
    float* u_old;        // NULL, or receives u before the step (gap iterations)
    float* ubar;         // plain N*N
    int* kt_clear;
    unsigned* qmax_next;
    const int* stop;
    int* iter;
};
struct WavGapArgs {
    int n, terms;
    const float* wu;     // W u
    KtView kt;
    const float* wtr;    // W^T r
    const float* u;
    const float* u_old;
    double* partials;
    const int* stop;
};
// the dual-tree complex wavelet transform (dtcwt.cu)
constexpr int CWT_MAX_TAPS = 16;
struct CwtBank {          // FP32 taps: level 1 (both trees), Q-shift tree a, Q-shift tree b
    int l1, lq;
    float h1[CWT_MAX_TAPS], g1[CWT_MAX_TAPS];
    float ha[CWT_MAX_TAPS], ga[CWT_MAX_TAPS];
    float hb[CWT_MAX_TAPS], gb[CWT_MAX_TAPS];
};
struct CwtGapArgs {
    int n, terms, ll_side;
    const float* tu;     // T planes of u (4 N^2)
    KtView kt;
    const float* wtr;    // W^T r
    const float* u;
    const float* u_old;
    double* partials;
    const int* stop;
};
int cwt_bank(const double* h1, int l1, const double* hq, int lq, CwtBank& bank, std::vector<double>* h1_out,
             std::vector<double>* hq_out);
void cwt_abs_sums(int n, int levels, const std::vector<double>& h1, const std::vector<double>& hq,
                  std::vector<double>& rows, std::vector<double>& cols);
// the DT-CWT's T planes (analysis) and its transpose; scratch: 5 N^2 / 4 floats per problem
int launch_cwt_analysis(const float* in, int N, int levels, const CwtBank& bank, float* out, float* scratch,
                        const int* stop, cudaStream_t st, int B, long long ps);
int launch_cwt_synthesis(float* in, int N, int levels, const CwtBank& bank, float* out, float* scratch,
                         const int* stop, cudaStream_t st, int B, long long ps);
int launch_cwt_dual(float* r, const float* T, const float* sig_r, const float* step_mul, const float* scal, int N,
                    int levels, const int* stop, cudaStream_t st, int B, long long ps);
int launch_cwt_uncombine(const float* r, float* T, int N, int levels, const int* stop, cudaStream_t st, int B,
                         long long ps);
int launch_cwt_gap_pixels(const CwtGapArgs& a, int nblocks, cudaStream_t st, int B, long long ps);
// the orthonormal Daubechies-4 transform (wavelet.cu)
bool wav_levels_ok(int n, int levels);
void wav_abs_sums(int n, int levels, std::vector<double>& rows, std::vector<double>& cols);
// The launches of the wavelet model cover B problems at once whose buffers (every pointer
// argument, the alpha/theta pair scal included) lie ps bytes apart; B = 1, ps = 0 for one.
int launch_wav_analysis(const float* in, int N, int levels, float* out, float* scratch, const int* stop, cudaStream_t st,
                        int B, long long ps);
int launch_wav_synthesis(const float* in, int N, int levels, float* out, float* scratch, const int* stop,
                         cudaStream_t st, int B, long long ps);
int launch_wav_dual(float* r, const float* wub, const float* sig_r, const float* step_mul, const float* scal,
                    long long nn, const int* stop, cudaStream_t st, int B, long long ps);
int launch_wav_primal(const WavPrimalArgs& a, cudaStream_t st, int B, long long ps);
int launch_wav_gap_pixels(const WavGapArgs& a, int nblocks, cudaStream_t st, int B, long long ps);
int launch_wav_tau(const float* kcol, const double* wcol, float* tau, long long nn, cudaStream_t st);

int ensure_precond(const pat_geometry* g, cudaStream_t st);
// y = K u for a plain N*N image (allocates its scratch from the stream-ordered pool)
int launch_forward(const pat_geometry* g, const float* u, float* y, cudaStream_t st);
// K^T y into an N*N float image (allocates its scratch from the stream-ordered pool).
int launch_adjoint(const pat_geometry* g, const float* y, float* out, cudaStream_t st);
KtView kt_view(const pat_geometry* g, const int* acc, const unsigned* ymax_bits);
// K^T y into an N*N float image using caller-provided, zeroed scratch (allocates nothing).
int launch_adjoint_into(const pat_geometry* g, const float* y, unsigned* ymax_bits, int* acc, float* out,
                        cudaStream_t st);


// max |y| as float bits into *out (which must hold 0 or a smaller value beforehand)
int launch_absmax(const float* y, long long n, unsigned* out, cudaStream_t st);

}  // namespace pat
