// 3x3 convolutions of the warm-start U-Net on the bfloat16 tensor cores (FP32 accumulate).
//
// Both kernels are implicit GEMMs staged through shared memory by a three-stage cp.async
// ring, with operands fed to mma.sync m16n8k16 (bf16 x bf16 -> f32) by ldmatrix.
//  - Forward (also the data gradient, with flipped weights): M = pixels, N = output
//    channels, K = 9 * input channels ordered (tap, channel), channels innermost.  A
//    16-byte vector of 8 channels never straddles a tap because the channel counts are
//    multiples of 8.  Out-of-image taps are zero-filled by the copy itself.
//  - Weight gradient: M = output channels, N = (tap, input channel), K = pixels.  Both
//    operands are stored pixel-major in memory and transposed by ldmatrix.trans.  The
//    pixel range is split over the grid's z dimension.  Each split writes its own partial
//    tile, and a second kernel sums the splits in a fixed order, so the result is
//    deterministic.
#include <algorithm>

#include "nn_internal.cuh"
#include "pat_internal.cuh"

namespace pat {
namespace nn {

namespace {

constexpr int STAGES = 3;
constexpr int THREADS = 256;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16-byte global -> shared copy; src_bytes = 0 writes zeros and reads nothing.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// d += a * b for one m16n8k16 tile (A row-major, B column-major fragments).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------------------
// forward: y[p][o] = bias[o] + sum_{tap, c} w[o][tap][c] x[p + tap][c]
// ---------------------------------------------------------------------------------------
constexpr int FBM = 128;          // pixels per CTA
constexpr int FBK = 32;           // K per stage
constexpr int FROW = FBK + 8;     // shared row stride (bf16): 80 bytes, conflict-free ldmatrix

struct FwdArgs {
    const bf16* x;
    int x_ps;
    const bf16* w;
    const float* bias;
    bf16* y;
    float* y32;
    int y_ps;
    int B, H, W, cin, cout, relu;
};

template <int BN, bool F32>
__global__ void __launch_bounds__(THREADS) k_conv_fwd(const FwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* sA = reinterpret_cast<bf16*>(smem);      // [STAGES][FBM][FROW]
    bf16* sB = sA + STAGES * FBM * FROW;          // [STAGES][BN][FROW]
    constexpr int WARPS_N = BN / 32;
    constexpr int WARPS_M = 8 / WARPS_N;
    constexpr int WM = FBM / WARPS_M;
    constexpr int MI = WM / 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp % WARPS_M, wn = warp / WARPS_M;
    const int HW = a.H * a.W;
    const long long P = (long long)a.B * HW;
    const long long m0 = (long long)blockIdx.x * FBM;
    const int n0 = blockIdx.y * BN;
    const int K = 9 * a.cin;
    const int nk = (K + FBK - 1) / FBK;

    // this thread copies 8-channel group g of rows (tid >> 2) + 64 i of the A tile
    const int g = tid & 3;
    int py[2], px[2];
    long long pimg[2];
    bool pok[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const long long p = m0 + (tid >> 2) + 64 * i;
        pok[i] = p < P;
        const long long pp = pok[i] ? p : 0;
        const int n = (int)(pp / HW), rem = (int)(pp - (long long)n * HW);
        py[i] = rem / a.W;
        px[i] = rem - py[i] * a.W;
        pimg[i] = (long long)n * HW;
    }

    auto load = [&](int stage, int kc) {
        const int k = kc * FBK + g * 8;
        const bool kok = k < K;
        const int tap = kok ? k / a.cin : 0;
        const int c = k - tap * a.cin;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        bf16* As = sA + stage * FBM * FROW;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = (tid >> 2) + 64 * i;
            const int yy = py[i] + dy, xx = px[i] + dx;
            const bool ok = kok && pok[i] && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const bf16* src = ok ? a.x + (pimg[i] + (long long)yy * a.W + xx) * a.x_ps + c : a.x;
            cp_async16(As + r * FROW + g * 8, src, ok ? 16 : 0);
        }
        bf16* Bs = sB + stage * BN * FROW;
#pragma unroll
        for (int j = 0; j < (BN + 63) / 64; ++j) {
            const int o = (tid >> 2) + 64 * j;
            if (o < BN) {
                const bool ok = kok && n0 + o < a.cout;
                const bf16* src = ok ? a.w + (size_t)(n0 + o) * K + k : a.w;
                cp_async16(Bs + o * FROW + g * 8, src, ok ? 16 : 0);
            }
        }
    };

    float acc[MI][4][4];
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) load(s, s);
        cp_async_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int st = kc % STAGES;
        const bf16* As = sA + st * FBM * FROW;
        const bf16* Bs = sB + st * BN * FROW;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t af[MI][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                const int row = wm * WM + mi * 16 + (lane & 15);
                const int col = ks * 16 + (lane >> 4) * 8;
                ldsm_x4(af[mi], As + row * FROW + col);
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int row = wn * 32 + nj * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int col = ks * 16 + ((lane >> 3) & 1) * 8;
                uint32_t t[4];
                ldsm_x4(t, Bs + row * FROW + col);
                bfr[2 * nj][0] = t[0];
                bfr[2 * nj][1] = t[1];
                bfr[2 * nj + 1][0] = t[2];
                bfr[2 * nj + 1][1] = t[3];
            }
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
        }
        const int nx = kc + STAGES - 1;
        if (nx < nk) load(nx % STAGES, nx);
        cp_async_commit();
    }
    cp_async_wait<0>();

    // epilogue: bias, ReLU, store (two adjacent channels per register pair)
#pragma unroll
    for (int mi = 0; mi < MI; ++mi) {
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int o = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
            if (o >= a.cout) continue;
            const float b0 = a.bias ? __ldg(a.bias + o) : 0.f;
            const float b1 = a.bias ? __ldg(a.bias + o + 1) : 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long p = m0 + wm * WM + mi * 16 + (lane >> 2) + 8 * h;
                if (p >= P) continue;
                float v0 = acc[mi][ni][2 * h] + b0, v1 = acc[mi][ni][2 * h + 1] + b1;
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (F32) {
                    *reinterpret_cast<float2*>(a.y32 + p * a.y_ps + o) = make_float2(v0, v1);
                } else {
                    *reinterpret_cast<__nv_bfloat162*>(a.y + p * a.y_ps + o) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// weight gradient: part[z][o][n] = sum over split z's pixels p of dz[p][o] x[p + tap(n)][c(n)]
// ---------------------------------------------------------------------------------------
constexpr int WBN = 128;   // (tap, channel) columns per CTA
constexpr int WBK = 32;    // pixels per stage

struct WgradArgs {
    const bf16* x;
    int x_ps;
    const bf16* dz;
    int dz_ps;
    float* part;      // [splits][cout][K]
    float* part_b;    // [splits][cout] or null
    int B, H, W, cin, cout;
    int chunks_per_split;
};

template <int BM>
__global__ void __launch_bounds__(THREADS) k_conv_wgrad(const WgradArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int SA = BM + 8, SB = WBN + 8;     // row strides (bf16): 16 mod 128 bytes
    bf16* sA = reinterpret_cast<bf16*>(smem);   // [STAGES][WBK][SA]  (pixel, out channel)
    bf16* sB = sA + STAGES * WBK * SA;          // [STAGES][WBK][SB]  (pixel, (tap, channel))
    constexpr int WARPS_M = BM / 32;
    constexpr int WARPS_N = 8 / WARPS_M;
    constexpr int WN = WBN / WARPS_N;
    constexpr int NI = WN / 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp % WARPS_M, wn = warp / WARPS_M;
    const int HW = a.H * a.W;
    const long long P = (long long)a.B * HW;
    const int K = 9 * a.cin;
    const int n0 = blockIdx.x * WBN, m0 = blockIdx.y * BM;
    const long long total_chunks = (P + WBK - 1) / WBK;
    const long long c_begin = (long long)blockIdx.z * a.chunks_per_split;
    const long long c_end = std::min<long long>(total_chunks, c_begin + a.chunks_per_split);
    const bool do_bias = a.part_b != nullptr && blockIdx.x == 0;

    auto load = [&](int stage, long long chunk) {
        const long long p0 = chunk * WBK;
        bf16* As = sA + stage * WBK * SA;
        constexpr int AV = WBK * BM / 8;         // 16-byte vectors of the A tile
        for (int v = tid; v < AV; v += THREADS) {
            const int row = v / (BM / 8), vg = v % (BM / 8);
            const long long p = p0 + row;
            const int o = m0 + vg * 8;
            const bool ok = p < P && o < a.cout;
            const bf16* src = ok ? a.dz + p * a.dz_ps + o : a.dz;
            cp_async16(As + row * SA + vg * 8, src, ok ? 16 : 0);
        }
        bf16* Bs = sB + stage * WBK * SB;
#pragma unroll
        for (int i = 0; i < WBK * WBN / 8 / THREADS; ++i) {
            const int v = tid + THREADS * i;
            const int row = v / (WBN / 8), vg = v % (WBN / 8);
            const long long p = p0 + row;
            const int n = n0 + vg * 8;
            bool ok = p < P && n < K;
            const bf16* src = a.x;
            if (ok) {
                const int tap = n / a.cin, c = n - tap * a.cin;
                const int img = (int)(p / HW), rem = (int)(p - (long long)img * HW);
                const int yy = rem / a.W + tap / 3 - 1, xx = rem % a.W + tap % 3 - 1;
                ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                if (ok) src = a.x + ((long long)img * HW + (long long)yy * a.W + xx) * a.x_ps + c;
            }
            cp_async16(Bs + row * SB + vg * 8, src, ok ? 16 : 0);
        }
    };

    float acc[2][NI][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
    float bsum = 0.f;

    const long long nk = c_end > c_begin ? c_end - c_begin : 0;
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) load(s, c_begin + s);
        cp_async_commit();
    }
    for (long long kc = 0; kc < nk; ++kc) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int st = (int)(kc % STAGES);
        const bf16* As = sA + st * WBK * SA;
        const bf16* Bs = sB + st * WBK * SB;
        if (do_bias && tid < BM) {
#pragma unroll 8
            for (int k = 0; k < WBK; ++k) bsum += __bfloat162float(As[k * SA + tid]);
        }
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int j = lane >> 3, r = lane & 7;
            uint32_t af[2][4], bfr[NI][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int k = ks * 16 + r + 8 * (j >> 1);
                const int m = wm * 32 + mi * 16 + 8 * (j & 1);
                ldsm_x4_t(af[mi], As + k * SA + m);
            }
#pragma unroll
            for (int nj = 0; nj < NI / 2; ++nj) {
                const int k = ks * 16 + r + 8 * (j & 1);
                const int n = wn * WN + nj * 16 + 8 * (j >> 1);
                uint32_t t[4];
                ldsm_x4_t(t, Bs + k * SB + n);
                bfr[2 * nj][0] = t[0];
                bfr[2 * nj][1] = t[1];
                bfr[2 * nj + 1][0] = t[2];
                bfr[2 * nj + 1][1] = t[3];
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
        }
        const long long nx = kc + STAGES - 1;
        if (nx < nk) load((int)(nx % STAGES), c_begin + nx);
        cp_async_commit();
    }
    cp_async_wait<0>();

    float* out = a.part + (size_t)blockIdx.z * a.cout * K;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int ni = 0; ni < NI; ++ni) {
            const int n = n0 + wn * WN + ni * 8 + (lane & 3) * 2;
            if (n >= K) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = m0 + wm * 32 + mi * 16 + (lane >> 2) + 8 * h;
                if (o < a.cout)
                    *reinterpret_cast<float2*>(out + (size_t)o * K + n) =
                        make_float2(acc[mi][ni][2 * h], acc[mi][ni][2 * h + 1]);
            }
        }
    }
    if (do_bias && tid < BM && m0 + tid < a.cout) a.part_b[(size_t)blockIdx.z * a.cout + m0 + tid] = bsum;
}

// out[i] = sum_z part[z][i] in the order z = 0, 1, ...
__global__ void k_sum_splits(const float* __restrict__ part, int splits, long long n, float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * n + i];
    out[i] = s;
}

__global__ void k_flip_weights(const bf16* __restrict__ w, int cout, int cin, bf16* __restrict__ wf) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)cout * 9 * cin;
    if (i >= n) return;
    // wf[c][t][o] = w[o][8 - t][c]
    const int o = (int)(i % cout);
    const int t = (int)((i / cout) % 9);
    const int c = (int)(i / ((long long)cout * 9));
    wf[i] = w[((size_t)o * 9 + (8 - t)) * cin + c];
}

template <int BN, bool F32>
int launch_fwd(const FwdArgs& a, cudaStream_t st) {
    const size_t smem = (size_t)STAGES * (FBM + BN) * FROW * sizeof(bf16);
    // a host-side attribute of the current device's function (no stream work; allowed
    // under graph capture)
    PAT_CUDA(cudaFuncSetAttribute(k_conv_fwd<BN, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long P = (long long)a.B * a.H * a.W;
    dim3 grid((unsigned)((P + FBM - 1) / FBM), (unsigned)((a.cout + BN - 1) / BN));
    k_conv_fwd<BN, F32><<<grid, THREADS, smem, st>>>(a);
    PAT_LAUNCH_CHECK("k_conv_fwd");
    return PAT_OK;
}

template <int BM>
int launch_wgrad(const WgradArgs& a, int splits, cudaStream_t st) {
    const size_t smem = (size_t)STAGES * WBK * ((BM + 8) + (WBN + 8)) * sizeof(bf16);
    const int K = 9 * a.cin;
    dim3 grid((unsigned)((K + WBN - 1) / WBN), (unsigned)((a.cout + BM - 1) / BM), (unsigned)splits);
    k_conv_wgrad<BM><<<grid, THREADS, smem, st>>>(a);
    PAT_LAUNCH_CHECK("k_conv_wgrad");
    return PAT_OK;
}

struct SplitPlan {
    int splits;
    long long per;
};

SplitPlan plan_splits(int B, int H, int W, int cin, int cout) {
    const long long P = (long long)B * H * W;
    const long long chunks = std::max<long long>(1, (P + WBK - 1) / WBK);
    const int bm = cout <= 32 ? 32 : 64;
    const long long tiles = (long long)((9 * cin + WBN - 1) / WBN) * ((cout + bm - 1) / bm);
    long long want = std::max<long long>(1, (2LL * sm_count() + tiles - 1) / tiles);
    want = std::min<long long>(want, std::max<long long>(1, chunks / 8));   // >= 8 chunks per split
    want = std::min<long long>(want, 512);
    const long long per = (chunks + want - 1) / want;
    return {(int)((chunks + per - 1) / per), per};
}

}  // namespace

int conv3x3_fwd(const View& x, int B, int H, int W, int cin, const bf16* w, const float* bias, int cout, bool relu,
                const View& y, float* y_f32, int y_f32_ps, cudaStream_t st) {
    if (B <= 0 || H <= 0 || W <= 0) return PAT_OK;
    FwdArgs a;
    a.x = x.p;
    a.x_ps = x.ps;
    a.w = w;
    a.bias = bias;
    a.y = y.p;
    a.y32 = y_f32;
    a.y_ps = y_f32 ? y_f32_ps : y.ps;
    a.B = B;
    a.H = H;
    a.W = W;
    a.cin = cin;
    a.cout = cout;
    a.relu = relu ? 1 : 0;
    if (y_f32) {
        if (cout <= 32) return launch_fwd<32, true>(a, st);
        if (cout <= 64) return launch_fwd<64, true>(a, st);
        return launch_fwd<128, true>(a, st);
    }
    if (cout <= 32) return launch_fwd<32, false>(a, st);
    if (cout <= 64) return launch_fwd<64, false>(a, st);
    return launch_fwd<128, false>(a, st);
}

size_t wgrad_partial_floats(int B, int H, int W, int cin, int cout) {
    const SplitPlan sp = plan_splits(B, H, W, cin, cout);
    return (size_t)sp.splits * cout * (9 * (size_t)cin + 1);
}

int conv3x3_wgrad(const View& x, const View& dz, int B, int H, int W, int cin, int cout, float* dw, float* db,
                  float* part, cudaStream_t st) {
    const SplitPlan sp = plan_splits(B, H, W, cin, cout);
    const long long nw = (long long)cout * 9 * cin;
    WgradArgs a;
    a.x = x.p;
    a.x_ps = x.ps;
    a.dz = dz.p;
    a.dz_ps = dz.ps;
    a.part = part;
    a.part_b = db ? part + (size_t)sp.splits * nw : nullptr;
    a.B = B;
    a.H = H;
    a.W = W;
    a.cin = cin;
    a.cout = cout;
    a.chunks_per_split = (int)sp.per;
    int rc = cout <= 32 ? launch_wgrad<32>(a, sp.splits, st) : launch_wgrad<64>(a, sp.splits, st);
    if (rc) return rc;
    k_sum_splits<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(part, sp.splits, nw, dw);
    PAT_LAUNCH_CHECK("k_sum_splits");
    if (db) {
        k_sum_splits<<<(unsigned)((cout + 255) / 256), 256, 0, st>>>(a.part_b, sp.splits, cout, db);
        PAT_LAUNCH_CHECK("k_sum_splits");
    }
    return PAT_OK;
}

int flip_weights(const bf16* w, int cout, int cin, bf16* wflip, cudaStream_t st) {
    const long long n = (long long)cout * 9 * cin;
    k_flip_weights<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, cout, cin, wflip);
    PAT_LAUNCH_CHECK("k_flip_weights");
    return PAT_OK;
}

}  // namespace nn
}  // namespace pat
