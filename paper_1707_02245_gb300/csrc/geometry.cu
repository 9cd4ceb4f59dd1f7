// Geometry creation, error reporting and small utilities of the C ABI.
//
// The discrete circular-mean operator (Sec. 4.2, eq. (K_def); Sec. 3.3.1): quadrature
// point m of circle (d, k) is x_d + r_k (cos phi_m, sin phi_m), phi_m = 2 pi (m + 1/2)/M,
// r_k = r0 + (k + 1/2) dr.  The tables built here are the only geometry state the
// kernels read: detector positions and the M (cos, sin) pairs (both scaled to pixel
// units), the FP32 radii (one FMA each, see radius()), arc weights 2 pi r_k / M, per
// group of 8 consecutive radii the circular range of angles whose points can touch the
// grid (a superset: kernels test every point exactly), and the K^T work list (ray
// segments per pixel tile and equal work items).
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <queue>
#include <vector>

#include "pat_internal.cuh"

namespace pat {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PAT_ERR_OOM : PAT_ERR_CUDA;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Streaming multiprocessors of the current device, queried once per device.
int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    const int slot = dev >= 0 && dev < 64 ? dev : 0;
    int n = cached[slot].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;   // no device: launch sizes only need a positive count
    }
    cached[slot].store(n, std::memory_order_relaxed);
    return n;
}

// ---- profiler --------------------------------------------------------------------
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mtx;
static double g_prof_ms[PAT_NPHASES];
static long long g_prof_n[PAT_NPHASES];

struct PendingMark {
    int phase;
    cudaEvent_t e0, e1;
};
static thread_local std::vector<cudaEvent_t> t_pool;
static thread_local std::vector<PendingMark> t_pending;
static thread_local size_t t_pool_used = 0;

static cudaEvent_t pool_event() {
    if (t_pool_used == t_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        t_pool.push_back(e);
    }
    return t_pool[t_pool_used++];
}

bool prof_on() { return g_prof.load(std::memory_order_relaxed); }

void prof_mark(int phase, cudaStream_t st, bool begin) {
    if (!prof_on()) return;
    cudaEvent_t e = pool_event();
    if (!e) return;
    cudaEventRecord(e, st);
    if (begin) {
        t_pending.push_back({phase, e, nullptr});
    } else {
        for (auto it = t_pending.rbegin(); it != t_pending.rend(); ++it)
            if (it->phase == phase && it->e1 == nullptr) {
                it->e1 = e;
                break;
            }
    }
}

void prof_collect() {
    if (t_pending.empty()) {
        t_pool_used = 0;
        return;
    }
    double ms[PAT_NPHASES] = {0};
    long long n[PAT_NPHASES] = {0};
    for (auto& m : t_pending) {
        float t = 0.f;
        if (m.e1 && cudaEventElapsedTime(&t, m.e0, m.e1) == cudaSuccess) {
            ms[m.phase] += t;
            n[m.phase] += 1;
        }
    }
    t_pending.clear();
    t_pool_used = 0;
    std::lock_guard<std::mutex> lock(g_prof_mtx);
    for (int i = 0; i < PAT_NPHASES; ++i) {
        g_prof_ms[i] += ms[i];
        g_prof_n[i] += n[i];
    }
}

}  // namespace pat

using namespace pat;

extern "C" int pat_profile_enable(int on) {
    g_prof.store(on != 0);
    return PAT_OK;
}

extern "C" int pat_profile_read(double* ms_host, long long* launches_host, int reset) {
    std::lock_guard<std::mutex> lock(g_prof_mtx);
    for (int i = 0; i < PAT_NPHASES; ++i) {
        if (ms_host) ms_host[i] = g_prof_ms[i];
        if (launches_host) launches_host[i] = g_prof_n[i];
        if (reset) {
            g_prof_ms[i] = 0;
            g_prof_n[i] = 0;
        }
    }
    return PAT_OK;
}

extern "C" long long pat_kernel_launches(void) { return g_launches.load(); }

extern "C" const char* pat_error_string(int code) {
    switch (code) {
        case PAT_OK: return "ok";
        case PAT_ERR_INVALID_ARG: return "invalid argument";
        case PAT_ERR_CUDA: return "CUDA error";
        case PAT_ERR_OOM: return "out of device memory";
        case PAT_ERR_NONFINITE: return "non-finite iterate or duality gap";
        case PAT_ERR_TIMEOUT: return "device-side wait timed out";
        default: return "unknown error";
    }
}

extern "C" const char* pat_last_error(void) { return g_last_error.c_str(); }

static void free_tables(pat_geometry* g) {
    cudaFree(g->det);
    cudaFree(g->cs);
    cudaFree(g->rk);
    cudaFree(g->wk);
    cudaFree(g->win);
    cudaFree(g->pc.krow);
    cudaFree(g->pc.kcol);
    cudaFree(g->pc.tile_kmax);
    cudaFree(g->adj_rays);
    cudaFree(g->adj_ray_geo);
    g->adj_ray_geo = nullptr;
    cudaFree(g->adj_item);
    cudaFree(g->fwd_units);
    cudaFree(g->fwd_ctas);
    cudaFree(g->fwd_roff);
    cudaFree(g->fwd_rgs);
    g->fwd_units = nullptr;
    g->fwd_ctas = nullptr;
    g->fwd_roff = nullptr;
    g->fwd_rgs = nullptr;
    g->adj_rays = nullptr;
    g->adj_item = nullptr;
    g->pc.tile_kmax = nullptr;
    g->det = nullptr;
    g->cs = nullptr;
    g->rk = nullptr;
    g->wk = nullptr;
    g->win = nullptr;
    g->pc.krow = nullptr;
    g->pc.kcol = nullptr;
}

// Smallest circular interval of [0, M) that covers every set entry of `mask`.
static int2 covering_window(const std::vector<unsigned char>& mask, int M) {
    int n_set = 0;
    for (int m = 0; m < M; ++m) n_set += mask[m];
    if (n_set == 0) return make_int2(0, 0);
    if (n_set == M) return make_int2(0, M);
    // longest circular run of unset entries; the window starts right after it
    int best_len = 0, best_end = 0;  // run occupies [best_end - best_len, best_end)
    int first_set = 0;
    while (!mask[first_set]) ++first_set;
    int run = 0;
    for (int s = 1; s <= M; ++s) {  // scan M entries starting after first_set
        int m = (first_set + s) % M;
        if (!mask[m]) {
            ++run;
        } else {
            if (run > best_len) {
                best_len = run;
                best_end = m;
            }
            run = 0;
        }
    }
    return make_int2(best_end, M - best_len);
}

// Checks a geometry description; returns PAT_OK or the error (with its message set).
static int check_desc(const pat_geometry_desc& d) {
    if (d.n < 2 || d.n > 16384) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: n must be in [2, 16384]");
    if (!(d.xmax > d.xmin) || !(d.ymax > d.ymin))
        return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: empty image extent");
    if (d.n_det < 1 || !d.det_xy_host) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: no detectors");
    if (d.n_t < 1) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: n_t must be >= 1");
    if (!(d.r0 >= 0.0) || !(d.dr > 0.0)) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: need r0 >= 0, dr > 0");
    if (d.quad_m < 1 || d.quad_m > MAX_QUAD_M)
        return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: quad_m must be in [1, 8192]");
    if ((long long)d.n_det * d.n_t > (1LL << 31) - 1)
        return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: D*T too large");
    for (int i = 0; i < 2 * d.n_det; ++i)
        if (!std::isfinite(d.det_xy_host[i])) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: non-finite detector");

    {
        // every quadrature point must have |fx|, |fy| < 2^22 (continuous pixel
        // coordinates), so the kernels' floors are exact and convert without clamping
        double ext = 0;
        const double rmax = d.r0 + d.n_t * d.dr;
        const double hx0 = (d.xmax - d.xmin) / d.n, hy0 = (d.ymax - d.ymin) / d.n;
        for (int i = 0; i < d.n_det; ++i) {
            ext = std::max(ext, (fabs(d.det_xy_host[2 * i] - d.xmin) + rmax) / hx0 + 1.0);
            ext = std::max(ext, (fabs(d.det_xy_host[2 * i + 1] - d.ymin) + rmax) / hy0 + 1.0);
        }
        if (!(ext < 4194304.0))
            return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: circles reach more than 2^22 pixels from the grid");
    }
    return PAT_OK;
}

// The FP32 device tables in continuous pixel coordinates (pixel centres at integers), and
// their FP64 counterparts (cos, sin of the angles; radii).
struct PointTables {
    std::vector<float2> det, cs;
    std::vector<float> rk, wk;
    std::vector<double> cosd, sind, rd;
};

static PointTables point_tables(const pat_geometry_desc& d) {
    const int N = d.n, D = d.n_det, T = d.n_t, M = d.quad_m;
    const double hx = (d.xmax - d.xmin) / N, hy = (d.ymax - d.ymin) / N;
    PointTables pt;
    pt.det.resize(D);
    pt.cs.resize(M);
    pt.rk.resize(T);
    pt.wk.resize(T);
    pt.cosd.resize(M);
    pt.sind.resize(M);
    pt.rd.resize(T);
    for (int i = 0; i < D; ++i)
        pt.det[i] = make_float2((float)((d.det_xy_host[2 * i] - d.xmin) / hx - 0.5),
                                (float)((d.det_xy_host[2 * i + 1] - d.ymin) / hy - 0.5));
    for (int m = 0; m < M; ++m) {
        const double phi = 2.0 * M_PI * (m + 0.5) / M;
        pt.cosd[m] = cos(phi);
        pt.sind[m] = sin(phi);
        pt.cs[m] = make_float2((float)(pt.cosd[m] / hx), (float)(pt.sind[m] / hy));
    }
    for (int k = 0; k < T; ++k) {
        pt.rd[k] = d.r0 + (k + 0.5) * d.dr;
        pt.rk[k] = radius(k, (float)d.dr, (float)(d.r0 + 0.5 * d.dr));
        pt.wk[k] = (float)(2.0 * M_PI * pt.rd[k] / M);
    }
    return pt;
}

// Two circular intervals of [0, M) that cover the set entries of mask: the complement of
// its two longest runs of unset entries.  Each is encoded m_first | count << 16.
static void cover_two(const unsigned char* mask, int M, unsigned& w0, unsigned& w1) {
    w0 = w1 = 0u;
    int first = -1, n_set = 0;
    for (int m = 0; m < M; ++m)
        if (mask[m]) {
            ++n_set;
            if (first < 0) first = m;
        }
    if (n_set == 0) return;
    if (n_set == M) {
        w0 = (unsigned)M << 16;
        return;
    }
    // runs of unset entries, in positions relative to `first` (a set entry)
    struct Run {
        int start, len;
    };
    Run best[2] = {{0, 0}, {0, 0}};
    int run_start = -1;
    for (int s = 1; s <= M; ++s) {   // position M is `first` again: it closes a trailing run
        const bool set = s == M || mask[(first + s) % M] != 0;
        if (!set) {
            if (run_start < 0) run_start = s;
        } else if (run_start >= 0) {
            const Run r{run_start, s - run_start};
            if (r.len > best[0].len) {
                best[1] = best[0];
                best[0] = r;
            } else if (r.len > best[1].len) {
                best[1] = r;
            }
            run_start = -1;
        }
    }
    if (best[1].len == 0) {   // one run of unset entries: one window, its complement
        const int s0 = best[0].start + best[0].len;
        w0 = (unsigned)((first + s0) % M) | ((unsigned)(M - best[0].len) << 16);
        return;
    }
    Run a = best[0], b = best[1];
    if (b.start < a.start) std::swap(a, b);
    const int s1 = a.start + a.len, c1 = b.start - s1;       // from the end of a to b
    const int s2 = b.start + b.len, c2 = a.start + M - s2;   // from the end of b round to a
    w0 = (unsigned)((first + s1) % M) | ((unsigned)c1 << 16);
    w1 = (unsigned)((first + s2) % M) | ((unsigned)c2 << 16);
}

struct SlabPlan {
    int slabs = 1, rows = 0, stride = 0, smem = 0;
    std::vector<int4> units;     // per CTA, round by round: {detector, window 0, window 1, k group << 16 | index}
    std::vector<int4> ctas;      // per CTA (cluster-major, rank-minor): {first rg entry, row groups, first roff entry, 0}
    std::vector<int> roff;       // per CTA: unit offsets of its rounds
    std::vector<int> rgs;        // per cluster: its row groups in processing order
    std::vector<float> cluster_cost;
    long long evaluated = 0;
};

// images above this side use the global-memory variant of K
// (on 16 x 512^2 batches the slab kernel, with its rounds of cluster barriers, measured
// slower than the global variant: 584 against 501 us per launch)
#ifndef PAT_FWD_SLAB_MAX_N
#define PAT_FWD_SLAB_MAX_N 320
#endif

// Slab count S (= CTAs per cluster) and rows R of geometry d for a K variant:
//  PAT_FWD_SLAB_TWO: the fewest slabs (at most FWD_MAX_CLUSTER) whose CTA fits two per SM;
//  PAT_FWD_SLAB_ONE: ... one per SM;
//  PAT_FWD_AUTO: the first of the two that fits, for images up to PAT_FWD_SLAB_MAX_N;
//  PAT_FWD_GLOBAL, or no slab shape fits: R = 0, the global-memory variant.
// budget_bytes > 0 instead caps the staged image of a slab (for tests).  With check, a
// shape whose clusters the device cannot hold is skipped.
static void slab_shape(const pat_geometry_desc& d, int budget_bytes, int& S, int& R, int& W, int& smem,
                       bool check = false, int variant = PAT_FWD_AUTO) {
    const int N = d.n, M = d.quad_m, D = d.n_det;
    W = (N + 6 + 3) / 4 * 4;   // columns -1 .. N + 1 at floats 3 .. N + 5
    if (W % 8 == 0) W += 4;   // W = 4 mod 8: 8 consecutive rows start in 8 different bank groups
    const bool staged = M <= FWD_STAGE_MAX && D <= FWD_STAGE_MAX &&
                        (variant != PAT_FWD_AUTO || N <= PAT_FWD_SLAB_MAX_N) && variant != PAT_FWD_GLOBAL;
    const int budgets[2] = {FWD_SMEM_TWO, FWD_SMEM_ONE};
    for (int bi = 0; bi < 2 && staged; ++bi) {
        if ((variant == PAT_FWD_SLAB_TWO && bi != 0) || (variant == PAT_FWD_SLAB_ONE && bi != 1)) continue;
        for (int s = 1; s <= FWD_MAX_CLUSTER; ++s) {
            const int r = (N + 1 + s - 1) / s;
            if (r < 8) break;
            const int need = forward_smem_bytes(r, W, M, D, true);
            const bool fits = budget_bytes > 0 ? (r + 1) * W * 4 <= budget_bytes && need <= FWD_SMEM_ONE
                                               : need <= budgets[bi];
            if (fits && (!check || forward_clusters_per_gpu(s, need) > 0)) {
                S = s;
                R = r;
                smem = need;
                return;
            }
        }
    }
    S = 1;
    R = 0;
    smem = forward_smem_bytes(0, W, M, D, false);
}

// The K work plan of geometry d for `n_clusters` clusters.
//  - Units: one per (row group, slab) with a point that can touch the grid in the slab,
//    covered by at most two angular windows.  Membership is decided in FP64 on the tables'
//    exact values with a margin of 1e-3 pixel, far above the FP32 rounding of a point's
//    position (about 1e-5 pixel), so every point the kernel counts in a slab lies inside
//    that slab's windows.
//  - Clusters: row groups dealt longest first onto the cluster whose slowest rank stays
//    least loaded; each cluster's list is shuffled (a fixed generator) so that every round
//    mixes detectors from all sides, and cut into rounds of FWD_ROUND.
static void build_slab_plan(const pat_geometry_desc& d, const PointTables& pt, const std::vector<int2>& win,
                            int n_clusters, int budget_bytes, SlabPlan& sp, int variant = PAT_FWD_AUTO,
                            bool check = false) {
    const int N = d.n, D = d.n_det, T = d.n_t, M = d.quad_m;
    const int n_kgrp = (T + KGRP - 1) / KGRP, n_rg = D * n_kgrp;
    const double hx = (d.xmax - d.xmin) / N, hy = (d.ymax - d.ymin) / N;
    int S, R, W, smem;
    slab_shape(d, budget_bytes, S, R, W, smem, check, variant);
    sp.slabs = S;
    sp.rows = R;
    sp.stride = W;
    sp.smem = smem;
    n_clusters = std::max(1, std::min(n_clusters, n_rg));
    const double eps = 1e-3;
    struct U {
        unsigned w0, w1;
        float cost;
    };
    // units[rg * S + s] (cost < 0: none)
    std::vector<U> units((size_t)n_rg * S, U{0u, 0u, -1.f});
    std::vector<unsigned char> mask((size_t)S * M);
    std::vector<char> touched(S);
    for (int di = 0; di < D; ++di) {
        const double px = (d.det_xy_host[2 * di] - d.xmin) / hx - 0.5;
        const double py = (d.det_xy_host[2 * di + 1] - d.ymin) / hy - 0.5;
        for (int gi = 0; gi < n_kgrp; ++gi) {
            const int rg = di * n_kgrp + gi;
            const int k0 = gi * KGRP, nk = std::min(T, k0 + KGRP) - k0;
            const int2 w = win[(size_t)rg];
            std::fill(touched.begin(), touched.end(), 0);
            for (int j = 0; j < w.y; ++j) {
                const int m = (w.x + j) % M;
                const double cx = pt.cosd[m] / hx, cy = pt.sind[m] / hy;
                for (int k = k0; k < k0 + nk; ++k) {
                    const double fx = px + pt.rd[k] * cx, fy = py + pt.rd[k] * cy;
                    if (!(fx > -1 - eps && fx < N + eps && fy > -1 - eps && fy < N + eps)) continue;
                    int s_lo = 0, s_hi = 0;
                    if (R > 0 && S > 1) {
                        s_lo = std::max(0, (int)std::floor((fy + 1 - eps) / R));
                        s_hi = std::min(S - 1, (int)std::floor((fy + 1 + eps) / R));
                    }
                    for (int s = s_lo; s <= s_hi; ++s) {
                        if (!touched[s]) {
                            touched[s] = 1;
                            std::fill(mask.begin() + (size_t)s * M, mask.begin() + (size_t)(s + 1) * M, 0);
                        }
                        mask[(size_t)s * M + m] = 1;
                    }
                }
            }
            for (int s = 0; s < S; ++s) {
                if (!touched[s]) continue;
                U& u = units[(size_t)rg * S + s];
                cover_two(&mask[(size_t)s * M], M, u.w0, u.w1);
                const long long pts = (long long)((u.w0 >> 16) + (u.w1 >> 16)) * nk;
                u.cost = (float)pts + 16.f;   // a unit's fixed work (fetch, phase sum)
                sp.evaluated += pts;
            }
        }
    }
    auto cost = [&](int rg, int s) { return std::max(0.f, units[(size_t)rg * S + s].cost); };
    // row groups to clusters
    std::vector<double> rg_total(n_rg, 0.0);
    for (int rg = 0; rg < n_rg; ++rg)
        for (int s = 0; s < S; ++s) rg_total[rg] += cost(rg, s);
    std::vector<int> order(n_rg);
    for (int i = 0; i < n_rg; ++i) order[i] = i;
    std::vector<double> load((size_t)n_clusters * S, 0.0);
    std::vector<std::vector<int>> members(n_clusters);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rg_total[x] > rg_total[y]; });
    for (int rg : order) {
        int best = 0;
        double best_max = 1e300;
        for (int c = 0; c < n_clusters; ++c) {
            double mx = 0.0;
            for (int s = 0; s < S; ++s) mx = std::max(mx, load[(size_t)c * S + s] + cost(rg, s));
            if (mx < best_max) {
                best_max = mx;
                best = c;
            }
        }
        for (int s = 0; s < S; ++s) load[(size_t)best * S + s] += cost(rg, s) + 1.0;   // + the epilogue
        members[best].push_back(rg);
    }
    unsigned long long lcg = 0x9E3779B97F4A7C15ull;
    for (int c = 0; c < n_clusters; ++c) {
        std::vector<int>& mem = members[c];
        if (mem.empty()) continue;
        std::sort(mem.begin(), mem.end());
        for (int i = (int)mem.size() - 1; i > 0; --i) {   // Fisher-Yates with a fixed LCG
            lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
            std::swap(mem[i], mem[(int)((lcg >> 33) % (unsigned long long)(i + 1))]);
        }
        const int rg0 = (int)sp.rgs.size();
        sp.rgs.insert(sp.rgs.end(), mem.begin(), mem.end());
        const int nrg = (int)mem.size(), n_rounds = (nrg + FWD_ROUND - 1) / FWD_ROUND;
        double worst = 0.0;
        for (int s = 0; s < S; ++s) {
            sp.ctas.push_back(make_int4(rg0, nrg, (int)sp.roff.size(), 0));
            double tot = 0.0;
            for (int rd = 0; rd < n_rounds; ++rd) {
                sp.roff.push_back((int)sp.units.size());
                std::vector<std::pair<float, int>> lst;   // (cost, index in the round)
                for (int i = rd * FWD_ROUND; i < std::min(nrg, (rd + 1) * FWD_ROUND); ++i)
                    if (units[(size_t)mem[i] * S + s].cost >= 0) lst.push_back({units[(size_t)mem[i] * S + s].cost, i});
                std::stable_sort(lst.begin(), lst.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
                for (auto& e : lst) {
                    const int rg = mem[e.second];
                    const U& u = units[(size_t)rg * S + s];
                    const int dd = rg / n_kgrp, kg = rg - dd * n_kgrp;
                    sp.units.push_back(make_int4(dd, (int)u.w0, (int)u.w1, (kg << 16) | (e.second - rd * FWD_ROUND)));
                    tot += e.first;
                }
            }
            sp.roff.push_back((int)sp.units.size());
            worst = std::max(worst, tot);
        }
        sp.cluster_cost.push_back((float)worst);
    }
}

struct AdjWork {
    int tiles_x = 0, tiles = 0;     // scale tiles
    int wtiles_x = 0, wtiles = 0;   // work tiles
    long long candidates = 0;
    std::vector<int4> rays;
    std::vector<AdjItem> items;
    std::vector<float> cost;
};

// The K^T work list of geometry d for a GPU that holds `slots` K^T CTAs at once.
static int adjoint_worklist(const pat_geometry_desc& d, const PointTables& pt, double slots, AdjWork& w,
                            int waves = ADJ_WAVES) {
    const int N = d.n, D = d.n_det, T = d.n_t, M = d.quad_m;
    const double hx = (d.xmax - d.xmin) / N, hy = (d.ymax - d.ymin) / N;
    const double ex = 1e-3 * hx, ey = 1e-3 * hy;
    const std::vector<float2>& det = pt.det;
    const std::vector<float2>& cs = pt.cs;
    // K^T candidate boxes: for every WTILE x WTILE work tile and detector, the (k, m)
    // polar box of the tile's tap region (points with i0 in [x0-1, x0+WTILE-1], same in
    // y), with one index of margin on every side; FP64 on the host
    w.tiles_x = (N + ATILE - 1) / ATILE;
    w.tiles = w.tiles_x * w.tiles_x;
    const int tiles_x = (N + WTILE - 1) / WTILE, tiles = tiles_x * tiles_x;
    w.wtiles_x = tiles_x;
    w.wtiles = tiles;
    std::vector<int4> box((size_t)tiles * D);
    for (int t = 0; t < tiles; ++t) {
        const int x0 = (t % tiles_x) * WTILE, y0 = (t / tiles_x) * WTILE;
        const double rx0 = d.xmin + (x0 - 0.5) * hx - ex, rx1 = d.xmin + (x0 + WTILE + 0.5) * hx + ex;
        const double ry0 = d.ymin + (y0 - 0.5) * hy - ey, ry1 = d.ymin + (y0 + WTILE + 0.5) * hy + ey;
        for (int di = 0; di < D; ++di) {
            const double dx = d.det_xy_host[2 * di], dy = d.det_xy_host[2 * di + 1];
            const double cx = std::min(std::max(dx, rx0), rx1), cy = std::min(std::max(dy, ry0), ry1);
            const double rmin = hypot(dx - cx, dy - cy);
            const double rmax = hypot(std::max(fabs(dx - rx0), fabs(dx - rx1)), std::max(fabs(dy - ry0), fabs(dy - ry1)));
            int k0 = (int)floor((rmin - d.r0) / d.dr - 0.5) - 1;
            int k1 = (int)ceil((rmax - d.r0) / d.dr - 0.5) + 1;
            k0 = std::max(k0, 0);
            k1 = std::min(k1, T - 1);
            int m0 = 0, nm = M;
            const bool inside = dx >= rx0 && dx <= rx1 && dy >= ry0 && dy <= ry1;
            if (!inside) {
                const double th0 = atan2(ry0 - dy, rx0 - dx);
                double lo = 0, hi = 0;
                const double px[3] = {rx1, rx0, rx1}, py[3] = {ry0, ry1, ry1};
                for (int c = 0; c < 3; ++c) {
                    double dth = atan2(py[c] - dy, px[c] - dx) - th0;
                    if (dth > M_PI) dth -= 2 * M_PI;
                    if (dth < -M_PI) dth += 2 * M_PI;
                    lo = std::min(lo, dth);
                    hi = std::max(hi, dth);
                }
                const double sc = M / (2 * M_PI);
                const long long mlo = (long long)floor((th0 + lo) * sc - 0.5) - 1;
                const long long mhi = (long long)ceil((th0 + hi) * sc - 0.5) + 1;
                if (mhi - mlo + 1 < M) {
                    nm = (int)(mhi - mlo + 1);
                    m0 = (int)(((mlo % M) + M) % M);
                }
            }
            if (k1 < k0) nm = 0;
            box[(size_t)t * D + di] = make_int4(k0, std::max(0, k1 - k0 + 1), m0, nm);
        }
    }

    // K^T work list.  Every ray (detector d, angle m) of a tile's polar box is cut to the
    // radius interval where its points can have taps in the tile's window [x0 - 1, x0 +
    // WTILE) x [y0 - 1, y0 + WTILE) (the window is convex, so the interval is one
    // segment).  The cut is FP64 arithmetic on the same FP32 tables the kernels read, on
    // the window widened by 1e-3 pixel, far beyond the FP32 rounding of a point's position
    // (about 1e-5 pixel); the kernel still tests every candidate exactly.  A tile's non-empty segments, concatenated, are its
    // candidate list: rays[] holds {d, m, first k, exclusive prefix} per segment and a
    // sentinel {-1, 0, 0, total} after each tile.  A work item (one CTA) is an equal share
    // of one tile's list; the shares are sized so that the items fill whole waves of the
    // GPU's resident CTAs.
    std::vector<int4>& rays = w.rays;
    std::vector<AdjItem>& items = w.items;
    std::vector<double> item_cost;
    {
        std::vector<long long> tile_base(tiles + 1, 0), tile_total(tiles, 0);
        for (int t = 0; t < tiles; ++t) {
            tile_base[t] = (long long)rays.size();
            const int x0 = (t % tiles_x) * WTILE, y0 = (t / tiles_x) * WTILE;
            const double wx0 = x0 - 1.001, wx1 = x0 + WTILE + 0.001;
            const double wy0 = y0 - 1.001, wy1 = y0 + WTILE + 0.001;
            long long pre = 0;
            for (int di = 0; di < D; ++di) {
                const int4 bx = box[(size_t)t * D + di];
                if (bx.w <= 0 || bx.y <= 0) continue;
                const long long kb = bx.x, ke = (long long)bx.x + bx.y;
                const double px = det[di].x, py = det[di].y;
                for (int j = 0; j < bx.w; ++j) {
                    const int m = (bx.z + j) % M;
                    const double cx = cs[m].x, cy = cs[m].y;
                    double t0 = -1e300, t1 = 1e300;
                    if (cx != 0) {
                        const double a0 = (wx0 - px) / cx, a1 = (wx1 - px) / cx;
                        t0 = std::max(t0, std::min(a0, a1));
                        t1 = std::min(t1, std::max(a0, a1));
                    } else if (px < wx0 || px > wx1) {
                        continue;
                    }
                    if (cy != 0) {
                        const double b0 = (wy0 - py) / cy, b1 = (wy1 - py) / cy;
                        t0 = std::max(t0, std::min(b0, b1));
                        t1 = std::min(t1, std::max(b0, b1));
                    } else if (py < wy0 || py > wy1) {
                        continue;
                    }
                    if (t1 < t0) continue;
                    const double kf0 = (t0 - d.r0) / d.dr - 0.5, kf1 = (t1 - d.r0) / d.dr - 0.5;
                    const long long k0 = (long long)std::max((double)kb, std::ceil(std::max(kf0, -1e15)));
                    const long long k1 = (long long)std::min((double)ke, std::floor(std::min(kf1, 1e15)) + 1);
                    if (k1 <= k0) continue;
                    rays.push_back(make_int4(di, m, (int)k0, (int)pre));
                    pre += k1 - k0;
                }
            }
            if (pre > (1LL << 30))
                return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: too many K^T candidates in one pixel tile");
            tile_total[t] = pre;
            rays.push_back(make_int4(-1, 0, 0, (int)pre));
        }
        tile_base[tiles] = (long long)rays.size();
        if (rays.size() > (size_t)((1LL << 31) - 1))
            return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: K^T work list too large");
        long long total = 0;
        for (int t = 0; t < tiles; ++t) total += tile_total[t];
        w.candidates = total;
        // pieces per tile: `waves` waves of resident CTAs (at least 1024 candidates a piece),
        // each piece going to the tile whose pieces are largest at that point, which
        // minimises the largest piece
        const long long Q = std::max(1LL, std::min((long long)(waves * slots), total / 1024));
        std::vector<long long> n_piece(tiles, 0);
        {
            std::priority_queue<std::pair<double, int>> heap;   // (piece size, tile)
            long long assigned = 0;
            for (int t = 0; t < tiles; ++t)
                if (tile_total[t] > 0) {
                    n_piece[t] = 1;
                    ++assigned;
                    heap.push({(double)tile_total[t], t});
                }
            for (; assigned < Q && !heap.empty(); ++assigned) {
                const int t = heap.top().second;
                heap.pop();
                ++n_piece[t];
                heap.push({(double)tile_total[t] / (double)n_piece[t], t});
            }
        }
        for (int t = 0; t < tiles; ++t) {
            const long long cost = tile_total[t];
            if (cost <= 0) continue;
            const long long n_p = n_piece[t];
            long long r = tile_base[t];                  // segment holding the piece's start
            for (long long j = 0; j < n_p; ++j) {
                long long b0 = cost * j / n_p;
                const long long b1 = cost * (j + 1) / n_p;
                if (b1 <= b0) continue;
                while (rays[r + 1].w <= b0) ++r;
                long long r_last = r;                    // segment holding b1 - 1
                while (rays[r_last + 1].w <= b1 - 1) ++r_last;
                while (b0 < b1) {                        // at most ARAYS segments per item
                    const long long re = std::min(r_last, r + ARAYS - 1);
                    const long long e1 = re == r_last ? b1 : rays[re + 1].w;
                    AdjItem it{};
                    it.tile = t;
                    it.ray0 = (int)r;
                    it.nray = (int)(re - r + 1);
                    it.c0 = (int)b0;
                    it.c1 = (int)e1;
                    items.push_back(it);
                    item_cost.push_back((double)(e1 - b0) + 4.0 * it.nray + 64.0);
                    b0 = e1;
                    if (b0 < b1) r = re + 1;
                }
            }
        }
        std::vector<int> order(items.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return item_cost[a] > item_cost[b]; });
        std::vector<AdjItem> sorted(items.size());
        w.cost.resize(items.size());
        for (size_t i = 0; i < order.size(); ++i) {
            sorted[i] = items[order[i]];
            w.cost[i] = (float)item_cost[order[i]];
        }
        items.swap(sorted);
        if (items.empty()) {   // one empty item keeps the launches well-formed
            AdjItem it{};
            it.ray0 = 0;
            items.push_back(it);
            w.cost.push_back(0.f);
        }
    }
    return PAT_OK;
}

// Angular windows of every (detector, group of KGRP radii): the smallest circular interval
// of angles whose points can touch the grid (FP64 with a margin of 1e-3 pixel).  Also
// counts the points whose taps touch the grid.
static std::vector<int2> grid_windows(const pat_geometry_desc& d, const PointTables& pt, long long* on_grid_out) {
    const int N = d.n, D = d.n_det, T = d.n_t, M = d.quad_m;
    const double hx = (d.xmax - d.xmin) / N, hy = (d.ymax - d.ymin) / N;
    const int n_kgrp = (T + KGRP - 1) / KGRP;
    const double ex = 1e-3 * hx, ey = 1e-3 * hy;
    const double xl = d.xmin - 0.5 * hx - ex, xh = d.xmax + 0.5 * hx + ex;
    const double yl = d.ymin - 0.5 * hy - ey, yh = d.ymax + 0.5 * hy + ey;
    const double gxl = d.xmin - 0.5 * hx, gxh = d.xmax + 0.5 * hx, gyl = d.ymin - 0.5 * hy, gyh = d.ymax + 0.5 * hy;
    std::vector<int2> win((size_t)D * n_kgrp);
    std::vector<unsigned char> mask(M);
    long long on_grid = 0;
    for (int di = 0; di < D; ++di) {
        const double dx = d.det_xy_host[2 * di], dy = d.det_xy_host[2 * di + 1];
        for (int gi = 0; gi < n_kgrp; ++gi) {
            std::fill(mask.begin(), mask.end(), 0);
            const int k_end = std::min(T, (gi + 1) * KGRP);
            for (int k = gi * KGRP; k < k_end; ++k) {
                const double r = pt.rd[k];
                const double cx = std::min(std::max(dx, xl), xh), cy = std::min(std::max(dy, yl), yh);
                const double dmin = hypot(dx - cx, dy - cy);
                const double dmax = std::max(std::max(hypot(dx - xl, dy - yl), hypot(dx - xh, dy - yl)),
                                             std::max(hypot(dx - xl, dy - yh), hypot(dx - xh, dy - yh)));
                if (r < dmin - 1e-9 || r > dmax + 1e-9) continue;
                for (int m = 0; m < M; ++m) {
                    const double x = dx + r * pt.cosd[m], y = dy + r * pt.sind[m];
                    if (x > gxl && x < gxh && y > gyl && y < gyh) ++on_grid;
                    if (!mask[m] && x > xl && x < xh && y > yl && y < yh) mask[m] = 1;
                }
            }
            win[(size_t)di * n_kgrp + gi] = covering_window(mask, M);
        }
    }
    if (on_grid_out) *on_grid_out = on_grid;
    return win;
}

// Builds the K plan of geometry g for `variant` and installs it (device arrays and view),
// replacing a previous plan.  The caller makes sure no work on g is in flight.
static int install_forward_plan(pat_geometry* g, const PointTables& pt, int variant) {
    const pat_geometry_desc& d = g->desc;
    pat_geometry_desc dd = d;
    dd.det_xy_host = g->det_xy.data();
    SlabPlan sp;
    {
        int S, R, W, smem;
        slab_shape(dd, 0, S, R, W, smem, true, variant);
        build_slab_plan(dd, pt, g->win_host, std::max(1, forward_clusters_per_gpu(S, smem)), 0, sp, variant, true);
    }
    int4 *units = nullptr, *ctas = nullptr;
    int *roff = nullptr, *rgs = nullptr;
    cudaError_t e = cudaSuccess;
    auto upload = [&](void** dst, const void* src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    upload((void**)&units, sp.units.data(), sizeof(int4) * sp.units.size());
    upload((void**)&ctas, sp.ctas.data(), sizeof(int4) * sp.ctas.size());
    upload((void**)&roff, sp.roff.data(), sizeof(int) * sp.roff.size());
    upload((void**)&rgs, sp.rgs.data(), sizeof(int) * sp.rgs.size());
    if (e != cudaSuccess) {
        cudaFree(units);
        cudaFree(ctas);
        cudaFree(roff);
        cudaFree(rgs);
        return cuda_fail(e, "K plan upload");
    }
    cudaFree(g->fwd_units);
    cudaFree(g->fwd_ctas);
    cudaFree(g->fwd_roff);
    cudaFree(g->fwd_rgs);
    g->fwd_units = units;
    g->fwd_ctas = ctas;
    g->fwd_roff = roff;
    g->fwd_rgs = rgs;
    g->points_per_apply = sp.evaluated;
    g->fwd_evaluated = sp.evaluated;
    g->fwd_cluster_cost = sp.cluster_cost;
    g->fwd_n_ctas = (int)sp.ctas.size();
    g->fwd_smem = sp.smem;
    g->shapes.forward = sp.rows > 0 ? (sp.smem <= FWD_SMEM_TWO ? PAT_FWD_SLAB_TWO : PAT_FWD_SLAB_ONE) : PAT_FWD_GLOBAL;
    GeomView& v = g->view;
    v.n_slabs = sp.slabs;
    v.slab_rows = sp.rows;
    v.slab_stride = sp.stride;
    v.smem_bytes = sp.smem;
    v.units = g->fwd_units;
    v.ctas = g->fwd_ctas;
    v.roff = g->fwd_roff;
    v.rgs = g->fwd_rgs;
    return PAT_OK;
}

// Builds the K^T work list of geometry g for work items that fill `waves` waves of
// resident CTAs and installs it, replacing a previous one.  No work on g may be in flight.
static int install_adjoint_plan(pat_geometry* g, const PointTables& pt, int waves) {
    pat_geometry_desc dd = g->desc;
    dd.det_xy_host = g->det_xy.data();
    AdjWork aw;
    const int rc = adjoint_worklist(dd, pt, (double)sm_count() * adjoint_blocks_per_sm(), aw, waves);
    if (rc) return rc;
    const std::vector<int4>& rays = aw.rays;
    const std::vector<AdjItem>& items = aw.items;
    // each segment's detector and direction next to it, so the K^T staging reads them in
    // one coalesced pass (sentinels get zeros)
    std::vector<float4> geo(rays.size());
    for (size_t i = 0; i < rays.size(); ++i)
        geo[i] = rays[i].x >= 0
                     ? make_float4(pt.det[rays[i].x].x, pt.det[rays[i].x].y, pt.cs[rays[i].y].x, pt.cs[rays[i].y].y)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    int4* r_dev = nullptr;
    float4* geo_dev = nullptr;
    AdjItem* it_dev = nullptr;
    cudaError_t e = cudaMalloc(&r_dev, sizeof(int4) * std::max<size_t>(rays.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(r_dev, rays.data(), sizeof(int4) * rays.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&geo_dev, sizeof(float4) * std::max<size_t>(geo.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(geo_dev, geo.data(), sizeof(float4) * geo.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&it_dev, sizeof(AdjItem) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(it_dev, items.data(), sizeof(AdjItem) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(r_dev);
        cudaFree(geo_dev);
        cudaFree(it_dev);
        return cuda_fail(e, "K^T work list upload");
    }
    cudaFree(g->adj_rays);
    cudaFree(g->adj_ray_geo);
    cudaFree(g->adj_item);
    g->adj_rays = r_dev;
    g->adj_ray_geo = geo_dev;
    g->adj_item = it_dev;
    g->adj_tiles_x = aw.tiles_x;
    g->adj_tiles = aw.tiles;
    g->adj_wtiles_x = aw.wtiles_x;
    g->adj_candidates = aw.candidates;
    g->adj_item_cost = aw.cost;
    g->adj_items = (int)items.size();
    g->shapes.adjoint_waves = waves;
    return PAT_OK;
}

extern "C" int pat_create_geometry(const pat_geometry_desc* desc, pat_geometry** out) {
    if (!desc || !out) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: NULL argument");
    *out = nullptr;
    const pat_geometry_desc& d = *desc;
    const int vrc = check_desc(d);
    if (vrc) return vrc;
    pat_geometry* g = new pat_geometry();
    g->desc = d;
    g->det_xy.assign(d.det_xy_host, d.det_xy_host + 2 * (size_t)d.n_det);
    g->desc.det_xy_host = nullptr;  // the caller's array is not retained
    cudaGetDevice(&g->device);

    const int N = d.n, D = d.n_det, T = d.n_t, M = d.quad_m;
    const int n_kgrp = (T + KGRP - 1) / KGRP;
    const PointTables pt = point_tables(d);

    // angular windows of every (detector, radius group) over the grid
    long long on_grid = 0;
    g->win_host = grid_windows(d, pt, &on_grid);
    g->points_on_grid = on_grid;
    const std::vector<int2>& win = g->win_host;

    cudaError_t e = cudaMalloc(&g->det, sizeof(float2) * D);
    if (e == cudaSuccess) e = cudaMalloc(&g->cs, sizeof(float2) * M);
    if (e == cudaSuccess) e = cudaMalloc(&g->rk, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&g->wk, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&g->win, sizeof(int2) * win.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->det, pt.det.data(), sizeof(float2) * D, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->cs, pt.cs.data(), sizeof(float2) * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->rk, pt.rk.data(), sizeof(float) * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->wk, pt.wk.data(), sizeof(float) * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->win, win.data(), sizeof(int2) * win.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "pat_create_geometry: table upload");
        free_tables(g);
        delete g;
        return rc;
    }
    GeomView& v = g->view;
    v.n = N;
    v.n_det = D;
    v.n_t = T;
    v.quad_m = M;
    v.n_kgrp = n_kgrp;
    v.det = g->det;
    v.cs = g->cs;
    v.rk = g->rk;
    v.wk = g->wk;
    v.dr_f = (float)d.dr;
    v.rh_f = (float)(d.r0 + 0.5 * d.dr);
    v.win = g->win;
    g->shapes.update_tile = PAT_UPD_32X4;
    int rc = install_forward_plan(g, pt, PAT_FWD_AUTO);
    if (!rc) rc = install_adjoint_plan(g, pt, ADJ_WAVES);
    if (rc) {
        free_tables(g);
        delete g;
        return rc;
    }
    *out = g;
    return PAT_OK;
}

extern "C" int pat_geometry_set_shapes(pat_geometry* g, const pat_shapes* s) {
    if (!g || !s) return fail(PAT_ERR_INVALID_ARG, "pat_geometry_set_shapes: NULL argument");
    if (s->forward < PAT_FWD_AUTO || s->forward > PAT_FWD_GLOBAL)
        return fail(PAT_ERR_INVALID_ARG, "pat_geometry_set_shapes: unknown K variant");
    if (s->adjoint_waves < 1 || s->adjoint_waves > 4)
        return fail(PAT_ERR_INVALID_ARG, "pat_geometry_set_shapes: adjoint_waves must be in [1, 4]");
    if (s->update_tile < PAT_UPD_32X4 || s->update_tile > PAT_UPD_64X4)
        return fail(PAT_ERR_INVALID_ARG, "pat_geometry_set_shapes: unknown update tile");
    int dev = 0;
    PAT_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(PAT_ERR_INVALID_ARG, "pat_geometry_set_shapes: the geometry belongs to another device");
    std::lock_guard<std::mutex> lock(g->mtx);
    PAT_CUDA(cudaDeviceSynchronize());   // the old plans may still be read by queued work
    pat_geometry_desc dd = g->desc;
    dd.det_xy_host = g->det_xy.data();
    const PointTables pt = point_tables(dd);
    // plans are rebuilt only when their shape changes (a rebuild re-evaluates every
    // quadrature point on the host)
    int rc = PAT_OK;
    if (s->forward != g->fwd_requested) {
        rc = install_forward_plan(g, pt, s->forward);
        if (!rc) g->fwd_requested = s->forward;
    }
    if (!rc && s->adjoint_waves != g->shapes.adjoint_waves) rc = install_adjoint_plan(g, pt, s->adjoint_waves);
    if (!rc) g->shapes.update_tile = s->update_tile;
    return rc;
}

extern "C" int pat_geometry_get_shapes(const pat_geometry* g, pat_shapes* s) {
    if (!g || !s) return fail(PAT_ERR_INVALID_ARG, "pat_geometry_get_shapes: NULL argument");
    *s = g->shapes;
    return PAT_OK;
}

extern "C" int pat_forward_plan(const pat_geometry_desc* desc, int budget_bytes, int sms, int* units_host,
                                long long units_cap, int* ctas_host, long long ctas_cap, int* roff_host,
                                long long roff_cap, int* rgs_host, long long rgs_cap, long long* info8_host) {
    if (!desc || !info8_host) return fail(PAT_ERR_INVALID_ARG, "pat_forward_plan: NULL argument");
    const int vrc = check_desc(*desc);
    if (vrc) return vrc;
    if (budget_bytes < 0 || budget_bytes > FWD_SMEM_ONE)
        return fail(PAT_ERR_INVALID_ARG, "pat_forward_plan: budget exceeds the K CTA's shared memory");
    int S, R, W, smem;
    slab_shape(*desc, budget_bytes, S, R, W, smem, sms <= 0);
    const int clusters = sms > 0 ? std::max(1, sms * (smem <= FWD_SMEM_TWO ? 2 : 1) / S)
                                 : std::max(1, forward_clusters_per_gpu(S, smem));
    const PointTables pt = point_tables(*desc);
    const std::vector<int2> win = grid_windows(*desc, pt, nullptr);
    SlabPlan sp;
    build_slab_plan(*desc, pt, win, clusters, budget_bytes, sp, PAT_FWD_AUTO, sms <= 0);
    info8_host[0] = sp.slabs;
    info8_host[1] = sp.rows;
    info8_host[2] = sp.stride;
    info8_host[3] = (long long)sp.units.size();
    info8_host[4] = (long long)sp.ctas.size();
    info8_host[5] = sp.evaluated;
    info8_host[6] = sp.smem;
    info8_host[7] = (long long)sp.roff.size();
    if ((units_host && units_cap < info8_host[3]) || (ctas_host && ctas_cap < info8_host[4]) ||
        (roff_host && roff_cap < info8_host[7]) || (rgs_host && rgs_cap < (long long)sp.rgs.size()))
        return fail(PAT_ERR_INVALID_ARG, "pat_forward_plan: output capacity too small");
    for (size_t i = 0; units_host && i < sp.units.size(); ++i) {
        units_host[4 * i] = sp.units[i].x;
        units_host[4 * i + 1] = sp.units[i].y;
        units_host[4 * i + 2] = sp.units[i].z;
        units_host[4 * i + 3] = sp.units[i].w;
    }
    for (size_t i = 0; ctas_host && i < sp.ctas.size(); ++i) {
        ctas_host[4 * i] = sp.ctas[i].x;
        ctas_host[4 * i + 1] = sp.ctas[i].y;
        ctas_host[4 * i + 2] = sp.ctas[i].z;
        ctas_host[4 * i + 3] = sp.ctas[i].w;
    }
    for (size_t i = 0; roff_host && i < sp.roff.size(); ++i) roff_host[i] = sp.roff[i];
    for (size_t i = 0; rgs_host && i < sp.rgs.size(); ++i) rgs_host[i] = sp.rgs[i];
    return PAT_OK;
}

extern "C" int pat_adjoint_worklist(const pat_geometry_desc* desc, int slots, int* rays_host, long long rays_cap,
                                    int* items_host, long long items_cap, long long* counts3_host) {
    if (!desc || !counts3_host) return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_worklist: NULL argument");
    const int vrc = check_desc(*desc);
    if (vrc) return vrc;
    double s = slots;
    if (slots <= 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return fail(PAT_ERR_CUDA, "pat_adjoint_worklist: no device to size the work list for (pass slots > 0)");
        }
        s = (double)sms * adjoint_blocks_per_sm();
    }
    AdjWork aw;
    const int rc = adjoint_worklist(*desc, point_tables(*desc), s, aw);
    if (rc) return rc;
    counts3_host[0] = (long long)aw.rays.size();
    counts3_host[1] = (long long)aw.items.size();
    counts3_host[2] = aw.candidates;
    if ((rays_host && rays_cap < counts3_host[0]) || (items_host && items_cap < counts3_host[1]))
        return fail(PAT_ERR_INVALID_ARG, "pat_adjoint_worklist: output capacity too small");
    if (rays_host)
        for (size_t i = 0; i < aw.rays.size(); ++i) {
            rays_host[4 * i] = aw.rays[i].x;
            rays_host[4 * i + 1] = aw.rays[i].y;
            rays_host[4 * i + 2] = aw.rays[i].z;
            rays_host[4 * i + 3] = aw.rays[i].w;
        }
    if (items_host)
        for (size_t i = 0; i < aw.items.size(); ++i) {
            const AdjItem& it = aw.items[i];
            int* o = items_host + 5 * i;
            o[0] = it.tile;
            o[1] = it.ray0;
            o[2] = it.nray;
            o[3] = it.c0;
            o[4] = it.c1;
        }
    return PAT_OK;
}

extern "C" void pat_destroy_geometry(pat_geometry* g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    free_tables(g);
    cudaSetDevice(cur);
    delete g;
}

extern "C" int pat_geometry_info(const pat_geometry* g, long long* out6) {
    if (!g || !out6) return fail(PAT_ERR_INVALID_ARG, "pat_geometry_info: NULL argument");
    out6[0] = g->desc.n;
    out6[1] = g->desc.n_det;
    out6[2] = g->desc.n_t;
    out6[3] = g->desc.quad_m;
    out6[4] = g->points_per_apply;
    out6[5] = g->points_on_grid;
    return PAT_OK;
}
