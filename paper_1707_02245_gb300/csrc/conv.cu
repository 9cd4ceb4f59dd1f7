// 3x3 convolutions of the warm-start U-Net on the bfloat16 tensor cores (FP32 accumulate).
//
// The forward pass (also the data gradient, with flipped weights) is an implicit GEMM with
// M = pixels, N = output channels, K = 9 * input channels ordered (tap, channel), channels
// innermost; a 16-byte vector of 8 channels never straddles a tap because the channel
// counts are multiples of 8.  It has two kernels, chosen by shape:
//  - k_conv_fwd_tc (64 or more input channels, or 32 in and more than 32 out): TMA boxes
//    into swizzled shared memory, tcgen05.mma with the accumulator in tensor memory,
//    warp-specialised and persistent (described at the kernel);
//  - k_conv_fwd (the narrow layers): a three-stage cp.async ring feeding mma.sync
//    m16n8k16 through ldmatrix; out-of-image taps are zero-filled by the copy itself.
// Weight gradient: k_conv_wgrad_tc (tcgen05; every layer with at most 256 output
// channels, described at the kernel), else k_conv_wgrad (mma.sync: M = output channels,
// N = (tap, input channel), K = pixels, the pixel-major operands transposed by
// ldmatrix.trans).  Both split the pixels; each split writes its own partial tile, and a
// second kernel sums the splits in a fixed order, so the result is deterministic.
#include <cuda.h>

#include <algorithm>
#include <mutex>

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
// forward on the 5th-generation tensor cores (tcgen05): a persistent, warp-specialised
// implicit GEMM  D[m][o] = sum_k A[m][k] B[o][k]  with the accumulator in tensor memory.
//   m: a pixel of a bx x by tile of one image (bx by = 128, bx a power of 2); o: an output
//   channel of an N tile of BN; k = (tap, channel), channels innermost.
// - warp 0 (one lane) is the TMA producer.  A stage holds K = 128 as 128 / CB boxes of CB
//   channels: for A the 4-D box {CB, bx, by, 1} of the NHWC activations at the tap's offset
//   (taps outside the image read TMA's zero fill), for B the 2-D box {CB, BN} of the
//   weights.  TMA writes them in the MMA's K-major layout, with the swizzle whose span is
//   the box's inner size (none for 16 bytes, else 32, 64 or 128 bytes).
// - warp 1 (one lane) issues tcgen05.mma (kind::f16: bf16 x bf16 -> f32, K = 16) into one
//   of four TMEM accumulators of BN columns, eight per stage (a wait on a barrier costs the
//   issuing thread about 300 cycles even when the phase is complete; eight MMAs amortise
//   it), and commits every stage to the stage's `empty` barrier and every finished tile to
//   its accumulator's `full` barrier.
// - warps 2..5 are the epilogue: warp w reads TMEM lanes 32 (w mod 4) + 0..31 (its pixels)
//   with tcgen05.ld, adds the bias, applies ReLU, stores 16-byte vectors and releases the
//   accumulator, so a tile's epilogue overlaps the next tile's loads and MMAs.
// One CTA per SM takes tiles round robin.  Every mbarrier wait gives up after about a
// second of SM clocks: the CTA counts a timeout in g_tc_timeouts, stops issuing, waits
// (again bounded) for its copies and MMAs in flight, frees its tensor memory and returns.
// ---------------------------------------------------------------------------------------
constexpr int TBM = 128;              // pixels per tile (TMEM lanes)
constexpr int TBK = 128;              // K per stage (eight MMAs per wait of the MMA thread)
constexpr int TC_THREADS = 192;       // producer warp, MMA warp, 4 epilogue warps
constexpr int TA_BYTES = TBM * TBK * 2;
constexpr long long T_WAIT_CYCLES = 2000000000LL;   // about 1 s at 2 GHz

__device__ unsigned int g_tc_timeouts;

struct TcArgs {
    int B, H, W, cin, cout, relu;
    int bx_log2, by;        // tile: 2^bx_log2 x by pixels
    int tiles_x, tiles_y, tiles_n, total;
    int cb;                 // channels per box: 8, 16, 32 or 64
    const float* bias;
    bf16* y;
    float* y32;
    int y_ps;
};

template <int BN>
struct TcCfg {
    static constexpr int STAGE = TA_BYTES + BN * TBK * 2;
    static constexpr int STAGES = BN == 128 ? 3 : (BN == 64 ? 4 : 5);
    static constexpr int NACC = 4;                                // TMEM accumulators (tiles in flight)
    static constexpr int BAR_OFF = STAGES * STAGE;               // full[S], empty[S], accf[NACC], acce[NACC], fin
    static constexpr int SLOT_OFF = BAR_OFF + 8 * (2 * STAGES + 2 * NACC + 1);
    static constexpr int SMEM = SLOT_OFF + 16 + 1024;            // + the 1024-byte alignment of the base
    static constexpr uint32_t NCOLS = NACC * BN;                 // a power of 2, at most 512
};

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// waits for the completion of phase `parity` of the barrier; false after the time limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > T_WAIT_CYCLES) return false;
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand: start, LBO and SBO in 16-byte
// units, descriptor version 1 (bits 46-47), base offset 0, layout (bits 61-63): 0 no
// swizzle, 6 = 32-byte, 4 = 64-byte, 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}

// instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the barrier completes a phase once every tcgen05.mma this thread issued before has finished
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (lane = thread)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    // the wait takes the registers as operands, so no use of them moves above it
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// tile t -> (image n, first pixel x0, y0, first output channel n0)
struct TcTile {
    int n, x0, y0, n0;
};
__device__ __forceinline__ TcTile tc_tile(const TcArgs& a, int t, int BN) {
    const int nt = t % a.tiles_n, mt = t / a.tiles_n;
    const int tx = mt % a.tiles_x, r = mt / a.tiles_x;
    TcTile q;
    q.x0 = tx << a.bx_log2;
    q.y0 = (r % a.tiles_y) * a.by;
    q.n = r / a.tiles_y;
    q.n0 = nt * BN;
    return q;
}

template <int BN, bool F32>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_fwd_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
    using C = TcCfg<BN>;
    constexpr int S = C::STAGES;
    constexpr uint32_t IDESC = tc_idesc(TBM, BN);
    static_assert(BN == 32 || BN == 64 || BN == 128, "N of the MMA");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bars = sbase + C::BAR_OFF;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (S + s); };
    constexpr int NA = C::NACC;
    auto accf = [&](int b) { return bars + 8u * (2 * S + b); };
    auto acce = [&](int b) { return bars + 8u * (2 * S + NA + b); };
    const uint32_t fin = bars + 8u * (2 * S + 2 * NA);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + C::SLOT_OFF);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::SLOT_OFF + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = 9 * a.cin, nk = (K + TBK - 1) / TBK;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < NA; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 4);   // one arrival per epilogue warp
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(C::NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicAdd(&g_tc_timeouts, 1u);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            int it = 0;
            const int q_per = TBK / a.cb;
            const uint32_t a_box = TBM * a.cb * 2, b_box = BN * a.cb * 2;
            for (int t = blockIdx.x; t < a.total && !*abort_flag; t += gridDim.x) {
                const TcTile tl = tc_tile(a, t, BN);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(empty(s), ((it / S) & 1) ^ 1)) {
                        give_up();
                        break;
                    }
                    mbar_expect_tx(full(s), (uint32_t)C::STAGE);
                    const uint32_t As = sbase + s * C::STAGE, Bs = As + TA_BYTES;
                    for (int q = 0; q < q_per; ++q) {
                        const int k = kc * TBK + q * a.cb;
                        int c = 0, x = 0, y = 0, n = a.B;   // past the last image: zero fill
                        if (k < K) {
                            const int tap = k / a.cin;
                            c = k - tap * a.cin;
                            x = tl.x0 + tap % 3 - 1;
                            y = tl.y0 + tap / 3 - 1;
                            n = tl.n;
                        }
                        tma_load_4d(As + q * a_box, &tmA, c, x, y, n, full(s));
                        tma_load_2d(Bs + q * b_box, &tmB, k, tl.n0, full(s));   // k >= K: zero fill
                    }
                }
            }
            // every copy issued has landed before the CTA may end (bounded)
            for (int j = it - 1; j >= 0 && j >= it - S; --j)
                if (!mbar_wait(full(j % S), (j / S) & 1)) {
                    give_up();
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            // descriptors without their start address, and each K step's byte offset in a stage
            const int cb = a.cb, lg = __ffs(cb) - 1;
            const uint32_t layout = cb == 8 ? 0u : cb == 16 ? 6u : cb == 32 ? 4u : 2u;
            const uint32_t a_reg = TBM * cb * 2, b_reg = BN * cb * 2;
            // no swizzle: LBO = the next 8 channels (next box region), SBO = the next 8 rows;
            // swizzled: SBO = one 8-row swizzle atom, LBO unused
            const uint32_t sbo = 8 * cb * 2;
            const uint64_t da = tc_desc(0, cb == 8 ? a_reg : 16, sbo, layout);
            const uint64_t db = tc_desc(0, cb == 8 ? b_reg : 16, sbo, layout);
            uint32_t a_off[TBK / 16], b_off[TBK / 16];
#pragma unroll
            for (int k16 = 0; k16 < TBK / 16; ++k16) {
                const int e = 16 * k16, reg = e >> lg;
                a_off[k16] = reg * a_reg + (uint32_t)((e & (cb - 1)) * 2);
                b_off[k16] = reg * b_reg + (uint32_t)((e & (cb - 1)) * 2);
            }
            int it = 0, tc = 0;
            for (int t = blockIdx.x; t < a.total && !*abort_flag; t += gridDim.x, ++tc) {
                const int b = tc % NA;
                if (!mbar_wait(acce(b), ((tc / NA) & 1) ^ 1)) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(full(s), (it / S) & 1)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t As = sbase + s * C::STAGE, Bs = As + TA_BYTES;
#pragma unroll
                    for (int k16 = 0; k16 < TBK / 16; ++k16)
                        tc_mma(d, da + ((As + a_off[k16]) >> 4), db + ((Bs + b_off[k16]) >> 4), IDESC, (kc | k16) != 0);
                    tc_commit(empty(s));
                }
                if (!ok) break;
                tc_commit(accf(b));
            }
            // every MMA issued has finished before the tensor memory is freed (bounded)
            tc_commit(fin);
            if (!mbar_wait(fin, 0)) give_up();
        }
    } else {
        // ---- epilogue: warps 2..5 ----
        const int quarter = warp & 3, row = quarter * 32 + lane;
        const int ly = row >> a.bx_log2, lx = row & ((1 << a.bx_log2) - 1);
        const uint32_t tl_lane = tmem + ((uint32_t)(quarter * 32) << 16);
        int tc = 0;
        for (int t = blockIdx.x; t < a.total; t += gridDim.x, ++tc) {
            const int b = tc % NA;
            int ok = 0;
            if (lane == 0) ok = mbar_wait(accf(b), (tc / NA) & 1) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) give_up();
                break;
            }
            tc_fence_after();
            const TcTile q = tc_tile(a, t, BN);
            const int y = q.y0 + ly, x = q.x0 + lx;
            const bool valid = y < a.H && x < a.W;
            const long long pp = ((long long)q.n * a.H + y) * a.W + x;
#pragma unroll
            for (int cb16 = 0; cb16 < BN / 16; ++cb16) {
                float v[16];
                __syncwarp();
                tc_ld16(tl_lane + (uint32_t)(b * BN + cb16 * 16), v);
                if (!valid) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int o = q.n0 + cb16 * 16 + 8 * h;
                    if (o >= a.cout) continue;   // cout is a multiple of 8
                    float w[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        w[e] = v[8 * h + e] + (a.bias ? __ldg(a.bias + o + e) : 0.f);
                        if (a.relu) w[e] = fmaxf(w[e], 0.f);
                    }
                    if (F32) {
                        float4* dst = reinterpret_cast<float4*>(a.y32 + pp * a.y_ps + o);
                        dst[0] = make_float4(w[0], w[1], w[2], w[3]);
                        dst[1] = make_float4(w[4], w[5], w[6], w[7]);
                    } else {
                        uint4 u;
                        __nv_bfloat162 t0 = __floats2bfloat162_rn(w[0], w[1]), t1 = __floats2bfloat162_rn(w[2], w[3]);
                        __nv_bfloat162 t2 = __floats2bfloat162_rn(w[4], w[5]), t3 = __floats2bfloat162_rn(w[6], w[7]);
                        u.x = *reinterpret_cast<uint32_t*>(&t0);
                        u.y = *reinterpret_cast<uint32_t*>(&t1);
                        u.z = *reinterpret_cast<uint32_t*>(&t2);
                        u.w = *reinterpret_cast<uint32_t*>(&t3);
                        *reinterpret_cast<uint4*>(a.y + pp * a.y_ps + o) = u;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(b));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::NCOLS) : "memory");
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

// ---------------------------------------------------------------------------------------
// weight gradient on the 5th-generation tensor cores: the same pipeline as k_conv_fwd_tc
// on the transposed problem  D[k][o] = sum_p X[p][k] dz[p][o],  k = (tap, channel) rows of
// an M tile of 128, o = the BN output channels, p = pixels (the GEMM's K) in tiles of PT
// (a wx x wy rectangle of one image, wx wy = PT).  Both operands are stored pixel-major,
// so both are MN-major for the MMA: TMA writes the box {CB channels, wx, wy, 1} of x at
// the tap's offset (zero fill outside the image) and the box {CBO channels, wx, wy, 1} of
// dz as rows of CB (CBO) channels per pixel, swizzled by the row size (32, 64 or 128
// bytes; 16-byte rows without swizzle).  An MN-major swizzle atom is 8 pixel rows; LBO
// steps from one channel box to the next, SBO from one 8-pixel group to the next (without
// swizzle the two swap).  A work unit is (M tile, split of the pixel
// tiles); the unit's partial D goes to part[split][o][k], summed over splits in a fixed
// order by k_sum_splits.
// ---------------------------------------------------------------------------------------
// pixels per stage: 128 (eight MMAs of K = 16 per wait) except at BN = 256 (64: the B tile
// of a stage is then 32 KB)
template <int BN>
constexpr int wg_pt() { return BN == 256 ? 64 : 128; }

struct WgTcArgs {
    int B, H, W, cin, cout;
    int wx_log2, wy;        // pixel tile: 2^wx_log2 x wy
    int ptiles_x, ptiles_y, n_ptiles;
    int m_tiles, splits, per, total;
    int cbx, cbo;           // channels per box of x and of dz: 8, 16, 32 or 64
    float* part;            // [splits][cout][9 cin]
};

template <int BN>
struct WgCfg {
    static constexpr int PT = wg_pt<BN>();
    static constexpr int A_BYTES = TBM * PT * 2;
    static constexpr int STAGE = A_BYTES + BN * PT * 2;
    static constexpr int STAGES = BN == 256 ? 4 : (BN == 128 ? 3 : 4);
    static constexpr int NACC = BN == 256 ? 2 : 4;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int SLOT_OFF = BAR_OFF + 8 * (2 * STAGES + 2 * NACC + 1);
    static constexpr int SMEM = SLOT_OFF + 16 + 1024;
    static constexpr uint32_t NCOLS = NACC * BN;
};

// instruction descriptor of kind::f16 with both operands MN-major (bits 15, 16)
constexpr uint32_t tc_idesc_mn(int M, int N) { return tc_idesc(M, N) | (1u << 15) | (1u << 16); }

// pixel tile pt -> its image and first pixel
__device__ __forceinline__ void wg_ptile(const WgTcArgs& a, int pt, int& n, int& x0, int& y0) {
    const int tx = pt % a.ptiles_x, r = pt / a.ptiles_x;
    x0 = tx << a.wx_log2;
    y0 = (r % a.ptiles_y) * a.wy;
    n = r / a.ptiles_y;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_wgrad_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmD, const WgTcArgs a) {
    using C = WgCfg<BN>;
    constexpr int S = C::STAGES, NA = C::NACC;
    constexpr uint32_t IDESC = tc_idesc_mn(TBM, BN);
    static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "N of the MMA");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bars = sbase + C::BAR_OFF;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (S + s); };
    auto accf = [&](int b) { return bars + 8u * (2 * S + b); };
    auto acce = [&](int b) { return bars + 8u * (2 * S + NA + b); };
    const uint32_t fin = bars + 8u * (2 * S + 2 * NA);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + C::SLOT_OFF);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::SLOT_OFF + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = 9 * a.cin;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < NA; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 4);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(C::NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    auto give_up = [&]() {
        *abort_flag = 1;
        atomicAdd(&g_tc_timeouts, 1u);
    };
    // the pixel tiles of unit u: [p_begin, p_end)
    auto unit_range = [&](int u, int& mt, int& p_begin, int& p_end) {
        mt = u % a.m_tiles;
        const int z = u / a.m_tiles;
        p_begin = z * a.per;
        p_end = min(a.n_ptiles, p_begin + a.per);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            int it = 0;
            const int qa = TBM / a.cbx, qb = BN / a.cbo;
            const uint32_t a_box = C::PT * a.cbx * 2, b_box = C::PT * a.cbo * 2;
            for (int u = blockIdx.x; u < a.total && !*abort_flag; u += gridDim.x) {
                int mt, pb, pe;
                unit_range(u, mt, pb, pe);
                for (int pt = pb; pt < pe; ++pt, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(empty(s), ((it / S) & 1) ^ 1)) {
                        give_up();
                        break;
                    }
                    mbar_expect_tx(full(s), (uint32_t)C::STAGE);
                    int n, x0, y0;
                    wg_ptile(a, pt, n, x0, y0);
                    const uint32_t As = sbase + s * C::STAGE, Bs = As + C::A_BYTES;
                    for (int q = 0; q < qa; ++q) {
                        const int k = mt * TBM + q * a.cbx;
                        int c = 0, x = 0, y = 0, nn = a.B;   // rows past K: zero fill
                        if (k < K) {
                            const int tap = k / a.cin;
                            c = k - tap * a.cin;
                            x = x0 + tap % 3 - 1;
                            y = y0 + tap / 3 - 1;
                            nn = n;
                        }
                        tma_load_4d(As + q * a_box, &tmX, c, x, y, nn, full(s));
                    }
                    for (int q = 0; q < qb; ++q)   // channels >= cout: zero fill
                        tma_load_4d(Bs + q * b_box, &tmD, q * a.cbo, x0, y0, n, full(s));
                }
            }
            for (int j = it - 1; j >= 0 && j >= it - S; --j)
                if (!mbar_wait(full(j % S), (j / S) & 1)) {
                    give_up();
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            // MN-major: LBO = the next channel box (next swizzle atom along M or N), SBO = the
            // next 8 pixel rows; a K step of 16 pixels advances two 8-row groups
            // Boxes of 8 channels (16-byte rows) use the MN-major layout without swizzle: an
            // 8 x 8 core matrix is 8 pixel rows of 16 bytes, the next 8 pixels 128 bytes on
            // (LBO), the next 8 channels one box on (SBO).
            auto desc = [&](int cb, uint32_t& kstep) -> uint64_t {
                if (cb == 8) {
                    kstep = 256;
                    return tc_desc(0, 128, C::PT * 16, 0u);
                }
                const uint32_t sbo = 8 * cb * 2;
                kstep = 2 * sbo;
                return tc_desc(0, C::PT * cb * 2, sbo, cb == 64 ? 2u : cb == 32 ? 4u : 6u);
            };
            uint32_t ks_a, ks_b;
            const uint64_t da = desc(a.cbx, ks_a), db = desc(a.cbo, ks_b);
            int it = 0, tc = 0;
            for (int u = blockIdx.x; u < a.total && !*abort_flag; u += gridDim.x, ++tc) {
                int mt, pb, pe;
                unit_range(u, mt, pb, pe);
                const int b = tc % NA;
                if (!mbar_wait(acce(b), ((tc / NA) & 1) ^ 1)) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                bool ok = true;
                for (int pt = pb; pt < pe; ++pt, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(full(s), (it / S) & 1)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t As = sbase + s * C::STAGE, Bs = As + C::A_BYTES;
#pragma unroll
                    for (int k16 = 0; k16 < C::PT / 16; ++k16)
                        tc_mma(d, da + ((As + k16 * ks_a) >> 4), db + ((Bs + k16 * ks_b) >> 4), IDESC,
                               (pt != pb || k16 != 0) ? 1u : 0u);
                    tc_commit(empty(s));
                }
                if (!ok) break;
                tc_commit(accf(b));
            }
            tc_commit(fin);
            if (!mbar_wait(fin, 0)) give_up();
        }
    } else {
        // ---- epilogue: warps 2..5; TMEM lane = row k of the M tile ----
        const int quarter = warp & 3, row = quarter * 32 + lane;
        const uint32_t tl_lane = tmem + ((uint32_t)(quarter * 32) << 16);
        int tc = 0;
        for (int u = blockIdx.x; u < a.total; u += gridDim.x, ++tc) {
            const int b = tc % NA;
            int ok = 0;
            if (lane == 0) ok = mbar_wait(accf(b), (tc / NA) & 1) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) give_up();
                break;
            }
            tc_fence_after();
            const int mt = u % a.m_tiles, z = u / a.m_tiles;
            const int k = mt * TBM + row;
            float* out = a.part + (size_t)z * a.cout * K;
#pragma unroll
            for (int cb16 = 0; cb16 < BN / 16; ++cb16) {
                float v[16];
                __syncwarp();
                tc_ld16(tl_lane + (uint32_t)(b * BN + cb16 * 16), v);
                if (k >= K) continue;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int o = cb16 * 16 + e;
                    if (o < a.cout) out[(size_t)o * K + k] = v[e];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce(b));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::NCOLS) : "memory");
    }
}

// part[g][o] = sum of dz[p][o] over the pixel range g of G equal ranges (a fixed order:
// 8-channel vectors by thread, rows strided by the block's row phases, then the phases in
// order)
__global__ void __launch_bounds__(256) k_colsum_part(const bf16* __restrict__ dz, int ps, long long P, int cout,
                                                     float* __restrict__ part) {
    __shared__ float sh[256][8];
    const int g = blockIdx.x, G = gridDim.x;
    const long long p0 = P * g / G, p1 = P * (g + 1) / G;
    const int nv = cout / 8, tid = threadIdx.x;
    const int phases = 256 / nv, v = tid % nv, ph = tid / nv;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ph < phases) {
        for (long long p = p0 + ph; p < p1; p += phases) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(dz + p * ps) + v);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h[e]);
                acc[2 * e] += f.x;
                acc[2 * e + 1] += f.y;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) sh[tid][e] = acc[e];
    __syncthreads();
    if (tid < nv) {
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int r = 0; r < phases; ++r)
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += sh[r * nv + tid][e];
#pragma unroll
        for (int e = 0; e < 8; ++e) part[(size_t)g * cout + tid * 8 + e] = s[e];
    }
}

// out[c] = sum_g part[g][c], one warp per column: lane l adds rows l, l + 32, ... in order,
// then a fixed butterfly over the lanes
__global__ void __launch_bounds__(256) k_sum_cols(const float* __restrict__ part, int rows, int cols,
                                                  float* __restrict__ out) {
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= cols) return;
    float s = 0.f;
    for (int g = lane; g < rows; g += 32) s += __ldg(part + (size_t)g * cols + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = s;
}

// out[i] = sum_z part[z][i]
__global__ void k_sum_splits(const float* __restrict__ part, int splits, long long n, float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // eight running sums (split z into sum z mod 8), added in order at the end: a fixed
    // order with eight loads in flight
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int z = 0;
    for (; z + 8 <= splits; z += 8)
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] += __ldg(part + (size_t)(z + j) * n + i);
    for (int j = 0; z < splits; ++z, ++j) s[j] += __ldg(part + (size_t)z * n + i);
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += s[j];
    out[i] = t;
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
    // a host-side attribute of the function (no stream work; allowed under graph capture),
    // set once
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_conv_fwd<BN, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    PAT_CUDA(attr);
    const long long P = (long long)a.B * a.H * a.W;
    dim3 grid((unsigned)((P + FBM - 1) / FBM), (unsigned)((a.cout + BN - 1) / BN));
    k_conv_fwd<BN, F32><<<grid, THREADS, smem, st>>>(a);
    PAT_LAUNCH_CHECK("k_conv_fwd");
    return PAT_OK;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, found once through the runtime (no link to libcuda)
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <int BN, bool F32>
int launch_fwd_tc(const FwdArgs& f, cudaStream_t st) {
    using C = TcCfg<BN>;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(PAT_ERR_CUDA, "conv3x3: cuTensorMapEncodeTiled is not available");
    TcArgs a;
    a.B = f.B;
    a.H = f.H;
    a.W = f.W;
    a.cin = f.cin;
    a.cout = f.cout;
    a.relu = f.relu;
    int lg = 0;
    while ((1 << lg) < f.W && lg < 7) ++lg;   // tile width: the power of 2 >= W, at most 128
    a.bx_log2 = lg;
    a.by = TBM >> lg;
    a.tiles_x = (f.W + (1 << lg) - 1) >> lg;
    a.tiles_y = (f.H + a.by - 1) / a.by;
    a.tiles_n = (f.cout + BN - 1) / BN;
    const long long total = (long long)f.B * a.tiles_x * a.tiles_y * a.tiles_n;
    if (total > (1LL << 30)) return fail(PAT_ERR_INVALID_ARG, "conv3x3: too many tiles");
    a.total = (int)total;
    a.cb = f.cin % 64 == 0 ? 64 : f.cin % 32 == 0 ? 32 : f.cin % 16 == 0 ? 16 : 8;
    a.bias = f.bias;
    a.y = f.y;
    a.y32 = f.y32;
    a.y_ps = f.y_ps;
    const CUtensorMapSwizzle sw = a.cb == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : a.cb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                  : a.cb == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                               : CU_TENSOR_MAP_SWIZZLE_NONE;
    // A: the NHWC activations as {channels, W, H, B} (pixel stride x_ps)
    CUtensorMap ma, mb;
    const cuuint64_t ps = (cuuint64_t)f.x_ps * 2;
    const cuuint64_t dA[4] = {(cuuint64_t)f.cin, (cuuint64_t)f.W, (cuuint64_t)f.H, (cuuint64_t)f.B};
    const cuuint64_t sA[3] = {ps, ps * f.W, ps * f.W * f.H};
    const cuuint32_t bA[4] = {(cuuint32_t)a.cb, (cuuint32_t)(1 << lg), (cuuint32_t)a.by, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)f.x, dA, sA, bA, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PAT_ERR_CUDA, "conv3x3: activation tensor map");
    // B: the weights as {K = 9 cin, cout}
    const int K = 9 * f.cin;
    const cuuint64_t dB[2] = {(cuuint64_t)K, (cuuint64_t)f.cout};
    const cuuint64_t sB[1] = {(cuuint64_t)K * 2};
    const cuuint32_t bB[2] = {(cuuint32_t)a.cb, (cuuint32_t)BN};
    r = enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)f.w, dB, sB, bB, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PAT_ERR_CUDA, "conv3x3: weight tensor map");
    // a host-side attribute of the function (allowed under graph capture), set once
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_conv_fwd_tc<BN, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    PAT_CUDA(attr);
    const int grid = (int)std::min<long long>(total, sm_count());
    k_conv_fwd_tc<BN, F32><<<grid, TC_THREADS, C::SMEM, st>>>(ma, mb, a);
    PAT_LAUNCH_CHECK("k_conv_fwd_tc");
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

constexpr int COLSUM_BLOCKS = 512;   // pixel ranges of the bias-gradient column sums

template <int BN>
int launch_wgrad_tc(const View& x, const View& dz, int B, int H, int W, int cin, int cout, float* dw, float* db,
                    float* part, int max_splits, cudaStream_t st) {
    using C = WgCfg<BN>;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(PAT_ERR_CUDA, "conv3x3_wgrad: cuTensorMapEncodeTiled is not available");
    WgTcArgs a;
    a.B = B;
    a.H = H;
    a.W = W;
    a.cin = cin;
    a.cout = cout;
    int lg = 0;
    while ((1 << lg) < W && (2 << lg) <= C::PT) ++lg;   // pixel tile width: the power of 2 >= W, at most PT
    a.wx_log2 = lg;
    a.wy = C::PT >> lg;
    a.ptiles_x = (W + (1 << lg) - 1) >> lg;
    a.ptiles_y = (H + a.wy - 1) / a.wy;
    const long long npt = (long long)B * a.ptiles_x * a.ptiles_y;
    const int K = 9 * cin;
    a.m_tiles = (K + TBM - 1) / TBM;
    if (npt > (1LL << 30)) return fail(PAT_ERR_INVALID_ARG, "conv3x3_wgrad: too many pixel tiles");
    a.n_ptiles = (int)npt;
    int splits = std::max(1, std::min(max_splits, (2 * sm_count() + a.m_tiles - 1) / a.m_tiles));
    a.per = (a.n_ptiles + splits - 1) / splits;
    a.splits = (a.n_ptiles + a.per - 1) / a.per;
    a.total = a.m_tiles * a.splits;
    auto box_ch = [](int c) { return c % 64 == 0 ? 64 : c % 32 == 0 ? 32 : c % 16 == 0 ? 16 : 8; };
    a.cbx = box_ch(cin);
    a.cbo = box_ch(cout);
    a.part = part;
    CUtensorMap mx, md;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    auto map4 = [&](CUtensorMap* m, const View& v, int ch, int cb) {
        const cuuint64_t ps = (cuuint64_t)v.ps * 2;
        const cuuint64_t dims[4] = {(cuuint64_t)ch, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {ps, ps * W, ps * W * H};
        const cuuint32_t box[4] = {(cuuint32_t)cb, (cuuint32_t)(1 << lg), (cuuint32_t)a.wy, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)v.p, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   cb == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                   : cb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                   : cb == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                              : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    if (map4(&mx, x, cin, a.cbx) != CUDA_SUCCESS) return fail(PAT_ERR_CUDA, "conv3x3_wgrad: activation tensor map");
    if (map4(&md, dz, cout, a.cbo) != CUDA_SUCCESS) return fail(PAT_ERR_CUDA, "conv3x3_wgrad: gradient tensor map");
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_conv_wgrad_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    PAT_CUDA(attr);
    k_conv_wgrad_tc<BN><<<std::min(a.total, sm_count()), TC_THREADS, C::SMEM, st>>>(mx, md, a);
    PAT_LAUNCH_CHECK("k_conv_wgrad_tc");
    const long long nw = (long long)cout * K;
    k_sum_splits<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(part, a.splits, nw, dw);
    PAT_LAUNCH_CHECK("k_sum_splits");
    if (db) {
        const long long P = (long long)B * H * W;
        const int G = (int)std::max<long long>(1, std::min<long long>(COLSUM_BLOCKS, (P + 63) / 64));
        float* pb = part + (size_t)a.splits * nw;
        k_colsum_part<<<G, 256, 0, st>>>(dz.p, dz.ps, P, cout, pb);
        PAT_LAUNCH_CHECK("k_colsum_part");
        k_sum_cols<<<(unsigned)((cout + 7) / 8), 256, 0, st>>>(pb, G, cout, db);
        PAT_LAUNCH_CHECK("k_sum_cols");
    }
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
    // The tensor-memory kernel wins where a pixel's channels fill 64-byte or 128-byte TMA
    // rows and the GEMM is wide enough (measured at batch 8: 1.6-2.5x for 64 or more input
    // channels); with 8-24 input channels, or 32 in and at most 32 out, the warp-level
    // kernel is as fast or faster (its loads are not bound by TMA's row rate).
    const bool tc = cin % 32 == 0 && (cin >= 64 || cout >= 64);
    if (y_f32) {
        if (cout <= 32) return tc ? launch_fwd_tc<32, true>(a, st) : launch_fwd<32, true>(a, st);
        if (cout <= 64) return tc ? launch_fwd_tc<64, true>(a, st) : launch_fwd<64, true>(a, st);
        return tc ? launch_fwd_tc<128, true>(a, st) : launch_fwd<128, true>(a, st);
    }
    if (cout <= 32) return tc ? launch_fwd_tc<32, false>(a, st) : launch_fwd<32, false>(a, st);
    if (cout <= 64) return tc ? launch_fwd_tc<64, false>(a, st) : launch_fwd<64, false>(a, st);
    return tc ? launch_fwd_tc<128, false>(a, st) : launch_fwd<128, false>(a, st);
}

size_t wgrad_partial_floats(int B, int H, int W, int cin, int cout) {
    const SplitPlan sp = plan_splits(B, H, W, cin, cout);
    return (size_t)sp.splits * cout * (9 * (size_t)cin + 1) + (size_t)COLSUM_BLOCKS * cout;
}

int conv3x3_wgrad(const View& x, const View& dz, int B, int H, int W, int cin, int cout, float* dw, float* db,
                  float* part, cudaStream_t st) {
    const SplitPlan sp = plan_splits(B, H, W, cin, cout);
    // the tensor-memory kernel (every layer with at most 256 output channels)
    if (cout <= 256 && B > 0 && H > 0 && W > 0) {
        if (cout <= 32) return launch_wgrad_tc<32>(x, dz, B, H, W, cin, cout, dw, db, part, sp.splits, st);
        if (cout <= 64) return launch_wgrad_tc<64>(x, dz, B, H, W, cin, cout, dw, db, part, sp.splits, st);
        if (cout <= 128) return launch_wgrad_tc<128>(x, dz, B, H, W, cin, cout, dw, db, part, sp.splits, st);
        return launch_wgrad_tc<256>(x, dz, B, H, W, cin, cout, dw, db, part, sp.splits, st);
    }
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

unsigned wait_timeouts() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return ~0u;
    }
    return v;
}

int flip_weights(const bf16* w, int cout, int cin, bf16* wflip, cudaStream_t st) {
    const long long n = (long long)cout * 9 * cin;
    k_flip_weights<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, cout, cin, wflip);
    PAT_LAUNCH_CHECK("k_flip_weights");
    return PAT_OK;
}

}  // namespace nn
}  // namespace pat
