// Geometry creation, error reporting and small utilities of the C ABI.
//
// The discrete circular-mean operator (Sec. 4.2, eq. (K_def); Sec. 3.3.1): quadrature
// point m of circle (d, k) is x_d + r_k (cos phi_m, sin phi_m), phi_m = 2 pi (m + 1/2)/M,
// r_k = r0 + (k + 1/2) dr.  The tables built here are the only geometry state the
// kernels read: detector positions and the M (cos, sin) pairs (both scaled to pixel
// units), radii, arc weights
// 2 pi r_k / M, and per group of 8 consecutive radii the circular range of angles
// whose points can touch the grid (a superset: kernels test every point exactly).
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstring>
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
    cudaFree(g->adj_box);
    cudaFree(g->adj_units);
    cudaFree(g->adj_item);
    g->adj_box = nullptr;
    g->adj_units = nullptr;
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

extern "C" int pat_create_geometry(const pat_geometry_desc* desc, pat_geometry** out) {
    if (!desc || !out) return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: NULL argument");
    *out = nullptr;
    const pat_geometry_desc& d = *desc;
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
        // every quadrature point must have |fx|, |fy| < 2^24 (continuous pixel
        // coordinates), so the kernels convert them to integers without clamping
        double ext = 0;
        const double rmax = d.r0 + d.n_t * d.dr;
        const double hx0 = (d.xmax - d.xmin) / d.n, hy0 = (d.ymax - d.ymin) / d.n;
        for (int i = 0; i < d.n_det; ++i) {
            ext = std::max(ext, (fabs(d.det_xy_host[2 * i] - d.xmin) + rmax) / hx0 + 1.0);
            ext = std::max(ext, (fabs(d.det_xy_host[2 * i + 1] - d.ymin) + rmax) / hy0 + 1.0);
        }
        if (!(ext < 16777216.0))
            return fail(PAT_ERR_INVALID_ARG, "pat_create_geometry: circles reach more than 2^24 pixels from the grid");
    }
    pat_geometry* g = new pat_geometry();
    g->desc = d;
    g->det_xy.assign(d.det_xy_host, d.det_xy_host + 2 * (size_t)d.n_det);
    g->desc.det_xy_host = nullptr;  // the caller's array is not retained
    cudaGetDevice(&g->device);

    const int N = d.n, D = d.n_det, T = d.n_t, M = d.quad_m;
    const double hx = (d.xmax - d.xmin) / N, hy = (d.ymax - d.ymin) / N;
    const int n_kgrp = (T + KGRP - 1) / KGRP;

    std::vector<float2> det(D), cs(M);
    std::vector<float> rk(T), wk(T);
    std::vector<double> cosd(M), sind(M), rd(T);
    // device tables in continuous pixel coordinates (pixel centres at integers)
    for (int i = 0; i < D; ++i)
        det[i] = make_float2((float)((d.det_xy_host[2 * i] - d.xmin) / hx - 0.5),
                             (float)((d.det_xy_host[2 * i + 1] - d.ymin) / hy - 0.5));
    for (int m = 0; m < M; ++m) {
        const double phi = 2.0 * M_PI * (m + 0.5) / M;
        cosd[m] = cos(phi);
        sind[m] = sin(phi);
        cs[m] = make_float2((float)(cosd[m] / hx), (float)(sind[m] / hy));
    }
    for (int k = 0; k < T; ++k) {
        rd[k] = d.r0 + (k + 0.5) * d.dr;
        rk[k] = (float)rd[k];
        wk[k] = (float)(2.0 * M_PI * rd[k] / M);
    }

    // angular windows: a point can touch the grid iff fx, fy in (-1, N), i.e.
    // x in (xmin - hx/2, xmax + hx/2); the test uses a margin so fp32 rounding in the
    // kernels never meets a point outside its window that would touch the grid
    const double ex = 1e-3 * hx, ey = 1e-3 * hy;
    const double xl = d.xmin - 0.5 * hx - ex, xh = d.xmax + 0.5 * hx + ex;
    const double yl = d.ymin - 0.5 * hy - ey, yh = d.ymax + 0.5 * hy + ey;
    std::vector<int2> win((size_t)D * n_kgrp);
    std::vector<unsigned char> mask(M);
    long long pts = 0, on_grid = 0;
    const double gxl = d.xmin - 0.5 * hx, gxh = d.xmax + 0.5 * hx, gyl = d.ymin - 0.5 * hy, gyh = d.ymax + 0.5 * hy;
    for (int di = 0; di < D; ++di) {
        const double dx = d.det_xy_host[2 * di], dy = d.det_xy_host[2 * di + 1];
        for (int gi = 0; gi < n_kgrp; ++gi) {
            std::fill(mask.begin(), mask.end(), 0);
            const int k_end = std::min(T, (gi + 1) * KGRP);
            for (int k = gi * KGRP; k < k_end; ++k) {
                const double r = rd[k];
                // quick reject: circle entirely off the extended box
                const double cx = std::min(std::max(dx, xl), xh), cy = std::min(std::max(dy, yl), yh);
                const double dmin = hypot(dx - cx, dy - cy);
                const double dmax = std::max(std::max(hypot(dx - xl, dy - yl), hypot(dx - xh, dy - yl)),
                                             std::max(hypot(dx - xl, dy - yh), hypot(dx - xh, dy - yh)));
                if (r < dmin - 1e-9 || r > dmax + 1e-9) continue;
                for (int m = 0; m < M; ++m) {
                    const double x = dx + r * cosd[m], y = dy + r * sind[m];
                    if (x > gxl && x < gxh && y > gyl && y < gyh) ++on_grid;  // touches the grid
                    if (!mask[m] && x > xl && x < xh && y > yl && y < yh) mask[m] = 1;
                }
            }
            int2 w = covering_window(mask, M);
            win[(size_t)di * n_kgrp + gi] = w;
            pts += (long long)w.y * (k_end - gi * KGRP);
        }
    }
    g->points_per_apply = pts;
    g->points_on_grid = on_grid;

    // K^T candidate boxes: for every ATILE x ATILE pixel tile and detector, the (k, m)
    // polar box of the tile's tap region (points with i0 in [x0-1, x0+ATILE-1], same in
    // y), with one index of margin on every side; FP64 on the host
    const int tiles_x = (N + ATILE - 1) / ATILE, tiles = tiles_x * tiles_x;
    std::vector<int4> box((size_t)tiles * D);
    for (int t = 0; t < tiles; ++t) {
        const int x0 = (t % tiles_x) * ATILE, y0 = (t / tiles_x) * ATILE;
        const double rx0 = d.xmin + (x0 - 0.5) * hx - ex, rx1 = d.xmin + (x0 + ATILE + 0.5) * hx + ex;
        const double ry0 = d.ymin + (y0 - 0.5) * hy - ey, ry1 = d.ymin + (y0 + ATILE + 0.5) * hy + ey;
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
    g->adj_tiles_x = tiles_x;
    g->adj_tiles = tiles;

    // K^T work list.  A unit is up to 32 rays of one (tile, detector) box; its cost is the
    // number of candidate points on those rays (ray-segment lengths in the tile's tap
    // region) plus a fixed overhead.  Each tile's units are packed into work items of
    // roughly equal cost (one CTA each); items run heaviest first.
    std::vector<int4> units;       // {detector, first ray (circular), rays, box index}
    std::vector<int4> items;       // {tile, first unit, end unit, 0}
    std::vector<double> item_cost;
    {
        std::vector<double> ucost;
        std::vector<int> tile_first(tiles + 1, 0);
        const double r_first = d.r0 + 0.5 * d.dr;
        for (int t = 0; t < tiles; ++t) {
            tile_first[t] = (int)units.size();
            const int x0 = (t % tiles_x) * ATILE, y0 = (t / tiles_x) * ATILE;
            const double rx0 = d.xmin + (x0 - 0.5) * hx - ex, rx1 = d.xmin + (x0 + ATILE + 0.5) * hx + ex;
            const double ry0 = d.ymin + (y0 - 0.5) * hy - ey, ry1 = d.ymin + (y0 + ATILE + 0.5) * hy + ey;
            for (int di = 0; di < D; ++di) {
                const int4 bx = box[(size_t)t * D + di];
                if (bx.w <= 0 || bx.y <= 0) continue;
                const double dx = d.det_xy_host[2 * di], dy = d.det_xy_host[2 * di + 1];
                for (int mb = 0; mb < bx.w; mb += 32) {
                    const int nr = std::min(32, bx.w - mb);
                    double c = 16.0;
                    for (int j = 0; j < nr; ++j) {
                        const int m = (bx.z + mb + j) % M;
                        const double cx = cosd[m], sy = sind[m];
                        double t0 = -1e300, t1 = 1e300;
                        if (cx != 0) {
                            const double a0 = (rx0 - dx) / cx, a1 = (rx1 - dx) / cx;
                            t0 = std::max(t0, std::min(a0, a1));
                            t1 = std::min(t1, std::max(a0, a1));
                        } else if (dx < rx0 || dx > rx1) {
                            t1 = -1e300;
                        }
                        if (sy != 0) {
                            const double b0 = (ry0 - dy) / sy, b1 = (ry1 - dy) / sy;
                            t0 = std::max(t0, std::min(b0, b1));
                            t1 = std::min(t1, std::max(b0, b1));
                        } else if (dy < ry0 || dy > ry1) {
                            t1 = -1e300;
                        }
                        if (t1 < t0) continue;
                        const double k0 = std::max((double)bx.x, floor((t0 - r_first) / d.dr) - 1);
                        const double k1 = std::min((double)(bx.x + bx.y), ceil((t1 - r_first) / d.dr) + 2);
                        c += std::max(0.0, k1 - k0);
                    }
                    units.push_back(make_int4(di, (bx.z + mb) % M, nr, t * D + di));
                    ucost.push_back(c);
                }
            }
        }
        tile_first[tiles] = (int)units.size();
        double total = 0;
        for (double c : ucost) total += c;
        const double target = std::max(64.0, total / (8.0 * 152.0));
        for (int t = 0; t < tiles; ++t) {
            int u = tile_first[t];
            while (u < tile_first[t + 1]) {
                double c = 0;
                const int u0 = u;
                while (u < tile_first[t + 1] && (u == u0 || c + ucost[u] <= target)) c += ucost[u++];
                items.push_back(make_int4(t, u0, u, 0));
                item_cost.push_back(c);
            }
        }
        std::vector<int> order(items.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return item_cost[a] > item_cost[b]; });
        std::vector<int4> sorted(items.size());
        g->adj_item_cost.resize(items.size());
        for (size_t i = 0; i < order.size(); ++i) {
            sorted[i] = items[order[i]];
            g->adj_item_cost[i] = (float)item_cost[order[i]];
        }
        items.swap(sorted);
        if (items.empty()) {
            items.push_back(make_int4(0, 0, 0, 0));
            g->adj_item_cost.push_back(0.f);
        }
    }
    g->adj_items = (int)items.size();

    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&g->det, sizeof(float2) * D);
    if (e == cudaSuccess) e = cudaMalloc(&g->cs, sizeof(float2) * M);
    if (e == cudaSuccess) e = cudaMalloc(&g->rk, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&g->wk, sizeof(float) * T);
    if (e == cudaSuccess) e = cudaMalloc(&g->win, sizeof(int2) * win.size());
    if (e == cudaSuccess) e = cudaMalloc(&g->adj_box, sizeof(int4) * box.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->adj_box, box.data(), sizeof(int4) * box.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->adj_units, sizeof(int4) * std::max<size_t>(1, units.size()));
    if (e == cudaSuccess && !units.empty())
        e = cudaMemcpy(g->adj_units, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->adj_item, sizeof(int4) * items.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->adj_item, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->det, det.data(), sizeof(float2) * D, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->cs, cs.data(), sizeof(float2) * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->rk, rk.data(), sizeof(float) * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->wk, wk.data(), sizeof(float) * T, cudaMemcpyHostToDevice);
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
    v.win = g->win;
    *out = g;
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
