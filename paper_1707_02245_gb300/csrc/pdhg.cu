// PDHGM iteration (Sec. 3.3, Algorithms 1 and 2) for TV, TGV^2 and directional TV, the
// diagonal steps of Sec. 3.3.2 and the FP64 duality gap / residual of Sec. 3.3.3.
//
// Schedule of one iteration n (two global dependency points: K needs all of ubar, the
// primal step needs all of K^T q):
//   1. k_forward_prox     q^{n+1} = prox(q^n + Sigma_q K ubar^n)              (data rows)
//   2. k_adjoint_tiles    w = K^T q^{n+1}                                    (pixel tiles)
//   3. k_update<REG>      on a pixel tile with a one-pixel halo:
//        u^{n+1}, v^{n+1} from w, r^{n+1}, s^{n+1};  ubar, vbar by extrapolation;
//        then the dual step of the NEXT iteration r^{n+2}, s^{n+2} from ubar, vbar.
//      r and s do not depend on q, so advancing their update by half an iteration gives
//      exactly the iterates of Algorithm 2.  vbar is never stored.
// x = (u, v) and (r, s) are ping-pong buffers: iteration n reads set n%2 and writes set
// (n+1)%2, because tiles read their neighbours' old values in the halo.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pat_internal.cuh"
#include "reduce.cuh"
#include "stencil.cuh"

namespace pat {

// update tiles (pat_shapes.update_tile): {TX, TY} of PAT_UPD_32X4, PAT_UPD_32X8, PAT_UPD_64X4
constexpr int UPD_TILES = 3;
constexpr int upd_tx(int t) { return t == PAT_UPD_64X4 ? 64 : 32; }
constexpr int upd_ty(int t) { return t == PAT_UPD_32X8 ? 8 : 4; }

struct UpdateArgs {
    int n;
    float alpha, ab, gamma, theta;
    // scalar steps (SCALAR2 rule); < 0 selects the diagonal rule
    float sig2, tau;
    const float* tau_u;    // N*N (diagonal rule)
    const float* sig_r;    // N*N (dTV diagonal rule)
    const float* xi;       // 2*N*N (dTV)
    const float* step_mul; // {s, 1/s}: multipliers of every primal and dual step (device)
    KtView kt;             // K^T q of this iteration (fixed point)
    int* kt_clear;         // the other fixed-point buffer, cleared here for the next iteration
    unsigned* qmax_next;   // max |q| slot of the next iteration, reset here
    const float* x_in;     // u, v1, v2
    const unsigned short* xl_in;   // low words of the compensated primal pairs (u, v1, v2), bfloat16
    const float* y_in;     // r1, r2, s11, s22, s12
    float* x_out;
    unsigned short* xl_out;
    float* y_out;
    float* ubar;           // N*N: ubar for the next K
    const int* stop;
    int* iter;             // iteration counter (incremented once per launch)
    int tiles_x;           // tiles per row of the grid
};

__device__ __forceinline__ float ld_img(const float* __restrict__ p, int N, int gx, int gy) {
    return (gx >= 0 && gx < N && gy >= 0 && gy < N) ? __ldg(p + gy * N + gx) : 0.f;
}

// One PDHG primal step plus the following dual step on a TX x TY tile.
template <int REG, int TX, int TY>
__device__ __forceinline__ void update_tile(const UpdateArgs& a, const int bx, const int by, const bool first) {
    constexpr int LX = TX + 2, LY = TY + 2;   // tile plus one-pixel halo on each side
    const int N = a.n;
    const size_t NN = (size_t)N * N;
    const int x0 = bx * TX, y0 = by * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;

    __shared__ float s_r1m[LY][LX], s_r2m[LY][LX];   // r (dTV: D_xi r) masked for div
    __shared__ float s_r1[LY][LX], s_r2[LY][LX];     // r as stored (the V cells and the tile read it)
    __shared__ float s_ub[LY][LX];                   // ubar on U = tile + high halo
    __shared__ float s_un[TY][TX];                   // u^{n+1} (high word) on the tile
    __shared__ unsigned short s_unl[TY][TX];         // ... its low word (bfloat16)
    // TGV only (small arrays for TV / dTV)
    constexpr int VL = (REG == PAT_TGV) ? LY : 1;
    constexpr int VX = (REG == PAT_TGV) ? LX : 1;
    constexpr int VT = (REG == PAT_TGV) ? TY : 1;
    constexpr int VTX = (REG == PAT_TGV) ? TX : 1;
    __shared__ float s_s11[VL][VX], s_s22[VL][VX], s_s12[VL][VX];
    __shared__ float s_vb1[VL][VX], s_vb2[VL][VX];   // vbar on V = tile + low halo
    __shared__ float s_vn1[VT][VTX], s_vn2[VT][VTX];
    __shared__ unsigned short s_vnl1[VT][VTX], s_vnl2[VT][VTX];

    // plane pointers, formed once
    const float* u_in = a.x_in;
    const float* r1_in = a.y_in;
    const float* r2_in = a.y_in + NN;
    const float* s11_in = a.y_in + 2 * NN;
    const float* s22_in = a.y_in + 3 * NN;
    const float* s12_in = a.y_in + 4 * NN;
    const float* v1_in = a.x_in + NN;
    const float* v2_in = a.x_in + 2 * NN;
    const unsigned short* v1l_in = a.xl_in + NN;
    const unsigned short* v2l_in = a.xl_in + 2 * NN;
    const float* xi0_in = a.xi;
    const float* xi1_in = REG == PAT_DTV ? a.xi + NN : a.xi;
    constexpr int NCELL = (LX * LY + TX * TY - 1) / (TX * TY);   // staged cells per thread
    const float tmul = __ldg(a.step_mul), smul = __ldg(a.step_mul + 1);

    // fixed-point scales of the K^T tiles that the cells of U (tile + high halo) touch: the
    // tile's sides divide or are multiples of ATILE, so U spans ceil(T / ATILE) + 1 of them
    static_assert(ATILE % TX == 0 || TX % ATILE == 0, "update tiles align with K^T tiles in x");
    static_assert(ATILE % TY == 0 || TY % ATILE == 0, "update tiles align with K^T tiles in y");
    constexpr int KNX = (TX + ATILE - 1) / ATILE + 1, KNY = (TY + ATILE - 1) / ATILE + 1;
    __shared__ float s_kinv[KNY][KNX];
    if (tid < KNX * KNY) {
        const int ktx = x0 / ATILE + tid % KNX, kty = y0 / ATILE + tid / KNX;
        s_kinv[tid / KNX][tid % KNX] = (ktx * ATILE < N && kty * ATILE < N) ? a.kt.inv_scale(ktx, kty) : 0.f;
    }

    // ---- stage 1: dual fields on the tile plus halo -------------------------------
    // Stage 2 visits the same cells.  The 32 x 8 tile (chosen for batches out of L2, where
    // occupancy matters) recomputes their coordinates there; the other tiles keep them
    // (measured at 256^2: 5.21 against 5.58 us; out of L2 the extra registers cost more).
    constexpr bool KEEP = TY != 8;
    int cl[NCELL], cgi[NCELL];   // cell (ly << 8 | lx) or -1; its global index or -1 off the grid
#pragma unroll
    for (int kc = 0; kc < NCELL; ++kc) {
        const int c = tid + kc * TX * TY;
        cl[kc] = -1;
        cgi[kc] = -1;
        if (c >= LX * LY) break;
        const int lx = c % LX, ly = c / LX;
        const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        const bool in = gx >= 0 && gx < N && gy >= 0 && gy < N;
        const int gi = in ? gy * N + gx : 0;
        cl[kc] = (ly << 8) | lx;
        cgi[kc] = in ? gi : -1;
        float r1 = in ? __ldg(r1_in + gi) : 0.f;
        float r2 = in ? __ldg(r2_in + gi) : 0.f;
        s_r1[ly][lx] = r1;
        s_r2[ly][lx] = r2;
        if (REG == PAT_DTV) {
            const float xi0 = in ? __ldg(xi0_in + gy * N + gx) : 0.f;
            const float xi1 = in ? __ldg(xi1_in + gy * N + gx) : 0.f;
            float o0, o1;
            dxi_apply(xi0, xi1, a.gamma, r1, r2, o0, o1);
            r1 = o0;
            r2 = o1;
        }
        s_r1m[ly][lx] = (gx < N - 1) ? r1 : 0.f;
        s_r2m[ly][lx] = (gy < N - 1) ? r2 : 0.f;
        if (REG == PAT_TGV) {
            s_s11[ly][lx] = in ? __ldg(s11_in + gi) : 0.f;
            s_s22[ly][lx] = in ? __ldg(s22_in + gi) : 0.f;
            s_s12[ly][lx] = in ? __ldg(s12_in + gi) : 0.f;
        }
    }
    __syncthreads();

    // ---- stage 2: primal step and extrapolation on U (u) and V (v) ------------------
#pragma unroll
    for (int kc = 0; kc < NCELL; ++kc) {
        int lx, ly, gi;
        bool in;
        if (KEEP) {
            if (cl[kc] < 0) break;
            lx = cl[kc] & 0xff;
            ly = cl[kc] >> 8;
            in = cgi[kc] >= 0;
            gi = cgi[kc];
        } else {
            const int c = tid + kc * TX * TY;
            if (c >= LX * LY) break;
            lx = c % LX;
            ly = c / LX;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            in = gx >= 0 && gx < N && gy >= 0 && gy < N;
            gi = gy * N + gx;
        }
        const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (lx >= 1 && ly >= 1) {  // U: u^{n+1}, ubar
            float ub = 0.f;
            if (in) {
                const float divr = s_r1m[ly][lx] - s_r1m[ly][lx - 1] + s_r2m[ly][lx] - s_r2m[ly - 1][lx];
                // (every rounding spelled out: a halo cell's value must equal, bit for
                // bit, the one its own tile computes in another unrolled copy)
                const float w = __fmul_rn((float)__ldg(&a.kt.acc[gi]),
                                          s_kinv[gy / ATILE - y0 / ATILE][gx / ATILE - x0 / ATILE]);
                const float uo = __ldg(u_in + gi), uol = lo_decode(__ldg(a.xl_in + gi));
                const float tu = __fmul_rn(a.tau >= 0.f ? a.tau : __ldg(a.tau_u + gi), tmul);
                float un = uo, unl = uol;
                add_compensated(un, unl, -__fmul_rn(tu, __fsub_rn(w, divr)));
                const unsigned short unq = lo_encode(unl);   // the stored pair, used from here on
                unl = lo_decode(unq);
                ub = fmaf(a.theta, (un - uo) + (unl - uol), un + unl);
                if (lx <= TX && ly <= TY) {
                    s_un[ly - 1][lx - 1] = un;
                    s_unl[ly - 1][lx - 1] = unq;
                }
            }
            s_ub[ly][lx] = ub;
        }
        if (REG == PAT_TGV && lx <= TX && ly <= TY) {  // V: v^{n+1}, vbar
            float vb1 = 0.f, vb2 = 0.f;
            if (in) {
                const bool ax = gx < N - 1, by = gy < N - 1;
                // E^T s = (-d_x^+ s11 - d_y^+ s12 / sqrt2, -d_y^+ s22 - d_x^+ s12 / sqrt2)
                const float dx11 = ax ? s_s11[ly][lx + 1] - s_s11[ly][lx] : 0.f;
                const float dy12 = by ? s_s12[ly + 1][lx] - s_s12[ly][lx] : 0.f;
                const float dy22 = by ? s_s22[ly + 1][lx] - s_s22[ly][lx] : 0.f;
                const float dx12 = ax ? s_s12[ly][lx + 1] - s_s12[ly][lx] : 0.f;
                const float et1 = __fsub_rn(-dx11, __fmul_rn(dy12, kInvSqrt2f));
                const float et2 = __fsub_rn(-dy22, __fmul_rn(dx12, kInvSqrt2f));
                const float r1 = s_r1[ly][lx], r2 = s_r2[ly][lx];
                const float v1o = __ldg(v1_in + gi), v2o = __ldg(v2_in + gi);
                const float v1ol = lo_decode(__ldg(v1l_in + gi)), v2ol = lo_decode(__ldg(v2l_in + gi));
                const float t1 = __fmul_rn(a.tau >= 0.f ? a.tau : tau_v1_tgv(gx, gy, N), tmul);
                const float t2 = __fmul_rn(a.tau >= 0.f ? a.tau : tau_v2_tgv(gx, gy, N), tmul);
                float v1n = v1o, v1nl = v1ol, v2n = v2o, v2nl = v2ol;
                add_compensated(v1n, v1nl, -__fmul_rn(t1, __fsub_rn(et1, r1)));
                add_compensated(v2n, v2nl, -__fmul_rn(t2, __fsub_rn(et2, r2)));
                const unsigned short v1q = lo_encode(v1nl), v2q = lo_encode(v2nl);
                v1nl = lo_decode(v1q);
                v2nl = lo_decode(v2q);
                vb1 = fmaf(a.theta, (v1n - v1o) + (v1nl - v1ol), v1n + v1nl);
                vb2 = fmaf(a.theta, (v2n - v2o) + (v2nl - v2ol), v2n + v2nl);
                if (lx >= 1 && ly >= 1) {
                    s_vn1[ly - 1][lx - 1] = v1n;
                    s_vn2[ly - 1][lx - 1] = v2n;
                    s_vnl1[ly - 1][lx - 1] = v1q;
                    s_vnl2[ly - 1][lx - 1] = v2q;
                }
            }
            s_vb1[ly][lx] = vb1;
            s_vb2[ly][lx] = vb2;
        }
    }
    __syncthreads();

    // ---- stage 3: dual step of the next iteration on the tile, and the writes --------
    const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
    if (gx < N && gy < N) {
        const int gi = gy * N + gx;
        const bool ax = gx < N - 1, by = gy < N - 1;
        const float ub = s_ub[ly][lx];
        const float gu0 = ax ? s_ub[ly][lx + 1] - ub : 0.f;
        const float gu1 = by ? s_ub[ly + 1][lx] - ub : 0.f;
        float r1 = s_r1[ly][lx], r2 = s_r2[ly][lx];
        if (REG == PAT_TV) {
            const float sr = (a.sig2 >= 0.f ? a.sig2 : sig_r_tv(gx, gy, N)) * smul;
            r1 = fmaf(sr, gu0, r1);
            r2 = fmaf(sr, gu1, r2);
        } else if (REG == PAT_DTV) {
            const float sr = (a.sig2 >= 0.f ? a.sig2 : __ldg(a.sig_r + gi)) * smul;
            float o0, o1;
            dxi_apply(__ldg(xi0_in + gi), __ldg(xi1_in + gi), a.gamma, gu0, gu1, o0, o1);
            r1 = fmaf(sr, o0, r1);
            r2 = fmaf(sr, o1, r2);
        } else {
            const float sr = (a.sig2 >= 0.f ? a.sig2 : sig_r_tgv(gx, gy, N)) * smul;
            r1 = fmaf(sr, gu0 - s_vb1[ly][lx], r1);
            r2 = fmaf(sr, gu1 - s_vb2[ly][lx], r2);
        }
        proj2(r1, r2, a.alpha);
        a.y_out[gi] = r1;
        a.y_out[NN + gi] = r2;
        a.x_out[gi] = s_un[threadIdx.y][threadIdx.x];
        a.xl_out[gi] = s_unl[threadIdx.y][threadIdx.x];
        a.ubar[gi] = ub;
        if (REG == PAT_TGV) {
            // E vbar with d^- on the masked field
            const bool axm = gx >= 1, bym = gy >= 1;
            const float v1 = ax ? s_vb1[ly][lx] : 0.f, v1l = axm ? s_vb1[ly][lx - 1] : 0.f;
            const float v2 = by ? s_vb2[ly][lx] : 0.f, v2d = bym ? s_vb2[ly - 1][lx] : 0.f;
            const float v1y = by ? s_vb1[ly][lx] : 0.f, v1d = bym ? s_vb1[ly - 1][lx] : 0.f;
            const float v2x = ax ? s_vb2[ly][lx] : 0.f, v2l = axm ? s_vb2[ly][lx - 1] : 0.f;
            const float e11 = v1 - v1l;
            const float e22 = v2 - v2d;
            const float e12 = ((v1y - v1d) + (v2x - v2l)) * kInvSqrt2f;
            const float ss = (a.sig2 >= 0.f ? a.sig2 : sig_s_tgv(gx, gy, N)) * smul;
            float s11 = fmaf(ss, e11, s_s11[ly][lx]);
            float s22 = fmaf(ss, e22, s_s22[ly][lx]);
            float s12 = fmaf(ss, e12, s_s12[ly][lx]);
            proj3(s11, s22, s12, a.ab);
            a.y_out[2 * NN + gi] = s11;
            a.y_out[3 * NN + gi] = s22;
            a.y_out[4 * NN + gi] = s12;
            a.x_out[NN + gi] = s_vn1[threadIdx.y][threadIdx.x];
            a.x_out[2 * NN + gi] = s_vn2[threadIdx.y][threadIdx.x];
            a.xl_out[NN + gi] = s_vnl1[threadIdx.y][threadIdx.x];
            a.xl_out[2 * NN + gi] = s_vnl2[threadIdx.y][threadIdx.x];
        }
    }
    if (gx < N && gy < N) a.kt_clear[gy * N + gx] = 0;
    if (first && tid == 0) {
        if (a.iter) *a.iter += 1;
        *a.qmax_next = 0u;
    }
}

template <int REG, int TILE>
__global__ void __launch_bounds__(upd_tx(TILE) * upd_ty(TILE)) k_update_b(const UpdateArgs* __restrict__ args,
                                                                          const int2* __restrict__ map) {
    const int2 pm = map[blockIdx.x];
    // the arguments in shared memory: their fields are read throughout the tile (measured:
    // 6.08 -> 5.58 us per launch at 256^2 against reading them from global memory)
    __shared__ UpdateArgs sa;
    const UpdateArgs& a = stage_args(args, pm.x, sa);
    if (a.stop && *(volatile const int*)a.stop) return;
    update_tile<REG, upd_tx(TILE), upd_ty(TILE)>(a, pm.y % a.tiles_x, pm.y / a.tiles_x, pm.y == 0);
}

// Dual step r, s <- prox(r, s + Sigma (A_reg (ubar, vbar))) used once before the first
// iteration (the update kernel performs it for every later iteration).
struct DualArgs {
    int n;
    float alpha, ab, gamma, sig2;
    float smul;            // dual step multiplier 1/s
    const float* sig_r;
    const float* xi;
    const float* ubar;     // N*N
    const float* vbar;     // 2*N*N (TGV)
    const float* y_in;
    float* y_out;
};

template <int REG>
__global__ void k_dual_step(DualArgs a) {
    const int N = a.n;
    const size_t NN = (size_t)N * N;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= N || gy >= N) return;
    const int gi = gy * N + gx;
    const bool ax = gx < N - 1, by = gy < N - 1;
    const float ub = a.ubar[gi];
    const float gu0 = ax ? a.ubar[gi + 1] - ub : 0.f;
    const float gu1 = by ? a.ubar[gi + N] - ub : 0.f;
    float r1 = a.y_in[gi], r2 = a.y_in[NN + gi];
    if (REG == PAT_TV) {
        const float sr = (a.sig2 >= 0.f ? a.sig2 : sig_r_tv(gx, gy, N)) * a.smul;
        r1 = fmaf(sr, gu0, r1);
        r2 = fmaf(sr, gu1, r2);
    } else if (REG == PAT_DTV) {
        const float sr = (a.sig2 >= 0.f ? a.sig2 : a.sig_r[gi]) * a.smul;
        float o0, o1;
        dxi_apply(a.xi[gi], a.xi[NN + gi], a.gamma, gu0, gu1, o0, o1);
        r1 = fmaf(sr, o0, r1);
        r2 = fmaf(sr, o1, r2);
    } else {
        const float sr = (a.sig2 >= 0.f ? a.sig2 : sig_r_tgv(gx, gy, N)) * a.smul;
        r1 = fmaf(sr, gu0 - a.vbar[gi], r1);
        r2 = fmaf(sr, gu1 - a.vbar[NN + gi], r2);
    }
    proj2(r1, r2, a.alpha);
    a.y_out[gi] = r1;
    a.y_out[NN + gi] = r2;
    if (REG == PAT_TGV) {
        auto vb = [&](int c, int x, int y) -> float { return a.vbar[c * NN + y * N + x]; };
        const bool axm = gx >= 1, bym = gy >= 1;
        const float v1 = ax ? vb(0, gx, gy) : 0.f, v1l = axm ? vb(0, gx - 1, gy) : 0.f;
        const float v2 = by ? vb(1, gx, gy) : 0.f, v2d = bym ? vb(1, gx, gy - 1) : 0.f;
        const float v1y = by ? vb(0, gx, gy) : 0.f, v1d = bym ? vb(0, gx, gy - 1) : 0.f;
        const float v2x = ax ? vb(1, gx, gy) : 0.f, v2l = axm ? vb(1, gx - 1, gy) : 0.f;
        const float e11 = v1 - v1l, e22 = v2 - v2d, e12 = ((v1y - v1d) + (v2x - v2l)) * kInvSqrt2f;
        const float ss = (a.sig2 >= 0.f ? a.sig2 : sig_s_tgv(gx, gy, N)) * a.smul;
        float s11 = fmaf(ss, e11, a.y_in[2 * NN + gi]);
        float s22 = fmaf(ss, e22, a.y_in[3 * NN + gi]);
        float s12 = fmaf(ss, e12, a.y_in[4 * NN + gi]);
        proj3(s11, s22, s12, a.ab);
        a.y_out[2 * NN + gi] = s11;
        a.y_out[3 * NN + gi] = s22;
        a.y_out[4 * NN + gi] = s12;
    }
}

// ---------------------------------------------------------------------------------
// FP64 duality gap over pixels (Sec. 3.3.3, box-restricted reading)
// partials per block: {R1, R2, |K^T q - div r|_1, |E^T s - r|_1, |x - x_old|^2, |x_old|^2}
// ---------------------------------------------------------------------------------
constexpr int GAP_PIX_TERMS = 7;   // per-block sums of the pixel pass
constexpr int GAP_TERMS = GAP_DATA_TERMS + GAP_PIX_TERMS;

// Distance of g from the normal cone of the radius-ball at p: the cone is {0} inside the
// ball and the ray through p on its sphere (the dual residual of a ball-constrained dual).
__device__ __forceinline__ float cone_distance2(float g0, float g1, float p0, float p1, float radius) {
    const float np = sqrtf(p0 * p0 + p1 * p1);
    const float lam = np >= radius * (1.f - 1e-6f) && np > 0.f ? fmaxf(0.f, (g0 * p0 + g1 * p1) / np) : 0.f;
    return sqrtf(fmaxf(g0 * g0 + g1 * g1 - lam * lam, 0.f));
}
__device__ __forceinline__ float cone_distance3(float g0, float g1, float g2, float p0, float p1, float p2,
                                                float radius) {
    const float np = sqrtf(p0 * p0 + p1 * p1 + p2 * p2);
    const float lam =
        np >= radius * (1.f - 1e-6f) && np > 0.f ? fmaxf(0.f, (g0 * p0 + g1 * p1 + g2 * p2) / np) : 0.f;
    return sqrtf(fmaxf(g0 * g0 + g1 * g1 + g2 * g2 - lam * lam, 0.f));
}

struct GapArgs {
    int n;
    float alpha, ab;      // ball radii of r and s
    double gamma;
    const float* xi;
    const float* x;       // x^{n+1}
    const float* x_old;   // x^n (NULL: residual terms are zero)
    const float* y;       // r, s at the same evaluation (y^{n+1})
    KtView kt;            // K^T q^{n+1} (fixed point)
    double* partials;
    const int* stop;
    int nblocks;          // blocks of this problem's pixel pass
};

template <int REG>
__device__ __forceinline__ void gap_pixels_block(const GapArgs& a, const int lb) {
    const int N = a.n;
    const size_t NN = (size_t)N * N;
    const float gam = (float)a.gamma;
    const float alpha = a.alpha, ab = a.ab;
    // per-thread terms in FP32 (each thread covers few pixels); warp sums as FP32 pairs and
    // block sums in FP64: GB300's FP64 pipe runs at 1/64 of FP32, so FP64 is kept to one
    // warp per block
    // + the dual residual of the regulariser duals (distance of their argument from the
    // normal cone of the ball at r and s), for the adaptive balance
    float acc[GAP_PIX_TERMS] = {0, 0, 0, 0, 0, 0, 0};
    const int nthreads = a.nblocks * blockDim.x;
    auto X = [&](int c, int x, int y) -> float { return __ldg(a.x + c * NN + (size_t)y * N + x); };
    auto Yf = [&](int c, int x, int y) -> float { return __ldg(a.y + c * NN + (size_t)y * N + x); };
    // r masked for div (dTV: D_xi r), zero outside the grid
    auto rm = [&](int c, int x, int y) -> float {
        if (x < 0 || y < 0 || (c == 0 && x >= N - 1) || (c == 1 && y >= N - 1)) return 0.f;
        float r0 = Yf(0, x, y), r1 = Yf(1, x, y);
        if (REG == PAT_DTV) {
            float o0, o1;
            dxi_apply(__ldg(a.xi + (size_t)y * N + x), __ldg(a.xi + NN + (size_t)y * N + x), gam, r0, r1, o0, o1);
            r0 = o0;
            r1 = o1;
        }
        return c == 0 ? r0 : r1;
    };
    for (long long p = (long long)lb * blockDim.x + threadIdx.x; p < (long long)NN; p += nthreads) {
        const int gx = (int)(p % N), gy = (int)(p / N);
        const bool ax = gx < N - 1, by = gy < N - 1;
        const float u = X(0, gx, gy);
        float g0 = ax ? X(0, gx + 1, gy) - u : 0.f;
        float g1 = by ? X(0, gx, gy + 1) - u : 0.f;
        if (REG == PAT_DTV) {
            float o0, o1;
            dxi_apply(__ldg(a.xi + p), __ldg(a.xi + NN + p), gam, g0, g1, o0, o1);
            g0 = o0;
            g1 = o1;
        }
        if (REG == PAT_TGV) {
            g0 -= X(1, gx, gy);
            g1 -= X(2, gx, gy);
        }
        acc[0] += sqrtf(g0 * g0 + g1 * g1);
        acc[6] += cone_distance2(g0, g1, Yf(0, gx, gy), Yf(1, gx, gy), alpha);
        // box term of u: |K^T q - div r|; near convergence the two sides agree closely and
        // their FP32 difference is exact (Sterbenz), so FP32 keeps the term's precision
        const float divr = (rm(0, gx, gy) - rm(0, gx - 1, gy)) + (rm(1, gx, gy) - rm(1, gx, gy - 1));
        const float atu = a.kt.at(gx, gy, N) - divr;
        acc[2] += fabsf(atu);
        if (REG == PAT_TGV) {
            auto vm = [&](int c, int x, int y, bool mx) -> float {  // masked v for d^-
                if (x < 0 || y < 0 || (mx ? (x >= N - 1) : (y >= N - 1))) return 0.f;
                return X(1 + c, x, y);
            };
            const float e11 = vm(0, gx, gy, true) - vm(0, gx - 1, gy, true);
            const float e22 = vm(1, gx, gy, false) - vm(1, gx, gy - 1, false);
            const float e12 = ((vm(0, gx, gy, false) - vm(0, gx, gy - 1, false)) +
                               (vm(1, gx, gy, true) - vm(1, gx - 1, gy, true))) * kInvSqrt2f;
            acc[1] += sqrtf(e11 * e11 + e22 * e22 + e12 * e12);
            const float s11 = Yf(2, gx, gy), s22 = Yf(3, gx, gy), s12 = Yf(4, gx, gy);
            acc[6] += cone_distance3(e11, e22, e12, s11, s22, s12, ab);
            const float dx11 = ax ? Yf(2, gx + 1, gy) - s11 : 0.f;
            const float dy12 = by ? Yf(4, gx, gy + 1) - s12 : 0.f;
            const float dy22 = by ? Yf(3, gx, gy + 1) - s22 : 0.f;
            const float dx12 = ax ? Yf(4, gx + 1, gy) - s12 : 0.f;
            const float et1 = -dx11 - dy12 * kInvSqrt2f, et2 = -dy22 - dx12 * kInvSqrt2f;
            acc[3] += fabsf(et1 - Yf(0, gx, gy)) + fabsf(et2 - Yf(1, gx, gy));
        }
        if (a.x_old) {
            const int nc = REG == PAT_TGV ? 3 : 1;
            for (int c = 0; c < nc; ++c) {
                const float xn = X(c, gx, gy), xo = __ldg(a.x_old + c * NN + p);
                acc[4] += (xn - xo) * (xn - xo);
                acc[5] += xo * xo;
            }
        }
    }
    double dacc[GAP_PIX_TERMS];
    block_sum_pair<GAP_PIX_TERMS>(acc, dacc);
    if (threadIdx.x == 0)
        for (int c = 0; c < GAP_PIX_TERMS; ++c) a.partials[GAP_PIX_TERMS * lb + c] = dacc[c];
}


constexpr int GAP_FINAL_BLOCKS = 32;
constexpr int GAP_FINAL_THREADS = 32;   // one warp: the final sums are FP64, kept to few lanes

struct InfoDev {
    double primal, dual, gap, rel_gap, residual;
    int iters_done, status, stop, iter;
    unsigned qmax_bits[2];  // max |q| of iterations of each parity (float bits)
    unsigned final_ticket;  // blocks of k_gap_final done (the last one resets it)
    float step_mul[2];      // {s, 1/s}: primal and dual step multipliers
    int n_adjust;           // adaptive-balance adjustments so far
    double level2[GAP_FINAL_BLOCKS][GAP_TERMS];
};

struct FinalArgs {
    const double* data_part;
    int n_data;
    const double* pix_part;
    int n_pix;
    double alpha, beta, box_u, box_v, tol;
    int reg, adapt;
    InfoDev* info;
    int* batch_stopped;    // problems of the batch that have stopped (the host polls it)
};

// Adaptive primal-dual balance (residual balancing after Goldstein, Li, Yuan, Esser and
// Baraniuk 2015), in L1 norms at the evaluated state:
//  - primal residual |A^T y|_1 (G = 0, so A^T y = 0 at a solution);
//  - dual residual: |q - (Ku - f)|_1, plus the distance of grad u - v (dTV: D_xi grad u)
//    and of E v from the normal cones of the r- and s-balls.
// When one exceeds the other by more than BAL_DEAD, s (the primal step multiplier) moves
// toward balance by the square root of their ratio, clamped to a factor BAL_MAX_STEP.  The
// exponent decays by BAL_DECAY per adjustment, so s settles.
constexpr double BAL_DEAD = 2.0, BAL_MAX_STEP = 2.0, BAL_DECAY = 0.97, BAL_MIN = 1e-3, BAL_MAX = 1e3;

__device__ void balance_update(InfoDev* in, double primal_res, double dual_res) {
    if (!(primal_res > 0 && dual_res > 0)) return;
    const double rho = primal_res / dual_res;
    if (rho >= 1.0 / BAL_DEAD && rho <= BAL_DEAD) return;
    const double f = fmin(fmax(sqrt(rho), 1.0 / BAL_MAX_STEP), BAL_MAX_STEP);
    double s = (double)in->step_mul[0] * pow(f, pow(BAL_DECAY, (double)in->n_adjust));
    s = fmin(fmax(s, BAL_MIN), BAL_MAX);
    in->step_mul[0] = (float)s;
    in->step_mul[1] = (float)(1.0 / s);
    in->n_adjust += 1;
}

__device__ __forceinline__ void gap_evaluate(const FinalArgs& a, const double (&t)[GAP_TERMS]);

// Two-level FP64 reduction in a fixed order: each of GAP_FINAL_BLOCKS blocks sums a fixed
// strided subset of the partials, the last block to finish adds the block sums in index
// order and evaluates the gap, the residual and the stopping test.
__device__ __forceinline__ void gap_final_block(const FinalArgs& a, const int lb) {
    double acc[GAP_TERMS];
    for (int c = 0; c < GAP_TERMS; ++c) acc[c] = 0.0;
    const int stride = GAP_FINAL_BLOCKS * blockDim.x;
    for (int b = lb * blockDim.x + threadIdx.x; b < a.n_data; b += stride)
        for (int c = 0; c < GAP_DATA_TERMS; ++c) acc[c] += a.data_part[GAP_DATA_TERMS * b + c];
    for (int b = lb * blockDim.x + threadIdx.x; b < a.n_pix; b += stride)
        for (int c = 0; c < GAP_PIX_TERMS; ++c) acc[GAP_DATA_TERMS + c] += a.pix_part[GAP_PIX_TERMS * b + c];
    block_sum<GAP_TERMS>(acc);
    __shared__ bool s_last;
    InfoDev* in = a.info;
    if (threadIdx.x == 0) {
        for (int c = 0; c < GAP_TERMS; ++c) in->level2[lb][c] = acc[c];
        __threadfence();
        s_last = atomicAdd(&in->final_ticket, 1u) == GAP_FINAL_BLOCKS - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // warp c adds the block sums of component c with a shuffle tree (fixed order)
    __shared__ double s_tot[GAP_TERMS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < GAP_TERMS; c += blockDim.x >> 5) {
        double v = lane < GAP_FINAL_BLOCKS ? *(volatile double*)&in->level2[lane][c] : 0.0;
        v = warp_sum(v);
        if (lane == 0) s_tot[c] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    in->final_ticket = 0;
    double t[GAP_TERMS];
    for (int c = 0; c < GAP_TERMS; ++c) t[c] = s_tot[c];
    gap_evaluate(a, t);
}

// The gap, the residual and the stopping test from the summed terms (one thread).
__device__ __forceinline__ void gap_evaluate(const FinalArgs& a, const double (&t)[GAP_TERMS]) {
    InfoDev* in = a.info;
    const double res2 = t[0], q2 = t[1], qf = t[2], dres_q = t[3];
    const double r1 = t[4], r2 = t[5], bu = t[6], bv = t[7], dx2 = t[8], x2 = t[9], dres_rs = t[10];
    const double reg = a.reg == PAT_TGV ? r1 + a.beta * r2 : r1;
    const double primal = 0.5 * res2 + a.alpha * reg;
    const double dual = -(0.5 * q2 + qf) - a.box_u * bu - (a.reg == PAT_TGV ? a.box_v * bv : 0.0);
    const double gap = primal - dual;
    const double rel = primal > 0 ? gap / primal : (gap == 0 ? 0.0 : INFINITY);
    const double resid = x2 > 0 ? sqrt(dx2 / x2) : (dx2 == 0 ? 0.0 : INFINITY);
    in->primal = primal;
    in->dual = dual;
    in->gap = gap;
    in->rel_gap = rel;
    in->residual = resid;
    in->iters_done = in->iter;
    if (!isfinite(gap) || !isfinite(primal)) {
        in->status = PAT_STATUS_DIVERGED;
        in->stop = 1;
        if (a.batch_stopped) atomicAdd(a.batch_stopped, 1);
    } else if (a.tol > 0 && rel <= a.tol) {
        in->status = PAT_STATUS_CONVERGED;
        in->stop = 1;
        if (a.batch_stopped) atomicAdd(a.batch_stopped, 1);
    } else if (a.adapt == PAT_ADAPT_BALANCE) {
        balance_update(in, bu + (a.reg == PAT_TGV ? bv : 0.0), dres_q + dres_rs);
    }
}

__global__ void __launch_bounds__(GAP_FINAL_THREADS) k_gap_final_b(const FinalArgs* __restrict__ args, const int2* __restrict__ map) {
    const int2 pm = map[blockIdx.x];
    __shared__ FinalArgs sa;
    const FinalArgs& a = stage_args(args, pm.x, sa);
    if (*(volatile const int*)&a.info->stop) return;
    gap_final_block(a, pm.y);
}

// The gap's pixel pass with the final reduction in its last block: every block writes its
// partial sums; the last of a problem's blocks to finish (a ticket) adds all the problem's
// data and pixel partials in FP64 in a fixed order (thread t takes rows t, t + 256, ...,
// then a fixed shuffle and warp tree) and evaluates the gap and the stopping test.
template <int REG>
__global__ void __launch_bounds__(256) k_gap_pixels_final_b(const GapArgs* __restrict__ args,
                                                            const FinalArgs* __restrict__ fin,
                                                            const int2* __restrict__ map) {
    const int2 pm = map[blockIdx.x];
    __shared__ GapArgs sa;
    const GapArgs& a = stage_args(args, pm.x, sa);
    if (a.stop && *(volatile const int*)a.stop) return;
    gap_pixels_block<REG>(a, pm.y);
    __shared__ bool s_last;
    InfoDev* in = fin[pm.x].info;
    if (threadIdx.x == 0) {
        __threadfence();   // this block's partials before its ticket
        s_last = atomicAdd(&in->final_ticket, 1u) == (unsigned)(a.nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const FinalArgs f = fin[pm.x];
    double acc[GAP_TERMS];
#pragma unroll
    for (int c = 0; c < GAP_TERMS; ++c) acc[c] = 0.0;
    for (int b = threadIdx.x; b < f.n_data; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < GAP_DATA_TERMS; ++c) acc[c] += __ldcg(f.data_part + GAP_DATA_TERMS * b + c);
    for (int b = threadIdx.x; b < f.n_pix; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < GAP_PIX_TERMS; ++c) acc[GAP_DATA_TERMS + c] += __ldcg(f.pix_part + GAP_PIX_TERMS * b + c);
    block_sum<GAP_TERMS>(acc);
    if (threadIdx.x != 0) return;
    in->final_ticket = 0;
    gap_evaluate(f, acc);
}

// ---------------------------------------------------------------------------------
// steps (Sec. 3.3.2): tau_u, sigma_r (dTV) need the K sums and xi; computed in FP64
// ---------------------------------------------------------------------------------
struct StepArgs {
    int n, reg;
    double gamma;
    const float* kcol;
    const float* xi;
    float* tau_u;
    float* sig_r;
    float* sig_s;
    float* tau_v;
};

__global__ void k_steps_pixels(StepArgs a) {
    const int N = a.n;
    const size_t NN = (size_t)N * N;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= N || gy >= N) return;
    const int gi = gy * N + gx;
    const double A = gx < N - 1, B = gy < N - 1;
    const double cx = (double)((gx < N - 1) + (gx >= 1)), cy = (double)((gy < N - 1) + (gy >= 1));
    double col_u = (double)a.kcol[gi];
    double sr = 1.0;
    if (a.reg == PAT_DTV) {
        auto dm = [&](int x, int y, double& d00, double& d01, double& d11) {
            const double z0 = a.xi[y * N + x], z1 = a.xi[NN + y * N + x];
            d00 = 1.0 - a.gamma * z0 * z0;
            d01 = -a.gamma * z0 * z1;
            d11 = 1.0 - a.gamma * z1 * z1;
        };
        double d00, d01, d11;
        dm(gx, gy, d00, d01, d11);
        // rows c = 0, 1 at this pixel: D_c0 d_x^+ + D_c1 d_y^+
        const double row0 = fabs(d00) * A + fabs(d01) * B + fabs(d00 * A + d01 * B);
        const double row1 = fabs(d01) * A + fabs(d11) * B + fabs(d01 * A + d11 * B);
        const double mx = fmax(row0, row1);
        sr = mx > 0 ? 1.0 / mx : 1.0;
        col_u += fabs(d00 * A + d01 * B) + fabs(d01 * A + d11 * B);
        if (gx >= 1) {
            double e00, e01, e11;
            dm(gx - 1, gy, e00, e01, e11);
            col_u += fabs(e00) + fabs(e01);
        }
        if (gy >= 1) {
            double e00, e01, e11;
            dm(gx, gy - 1, e00, e01, e11);
            col_u += fabs(e01) + fabs(e11);
        }
    } else {
        col_u += cx + cy;
        if (a.reg == PAT_TV) {
            const double m = fmax(2 * A, 2 * B);
            sr = m > 0 ? 1.0 / m : 1.0;
        } else {
            sr = 1.0 / fmax(2 * A + 1, 2 * B + 1);
        }
    }
    if (a.tau_u) a.tau_u[gi] = (float)(1.0 / col_u);
    if (a.sig_r) a.sig_r[gi] = (float)sr;
    if (a.reg == PAT_TGV) {
        if (a.sig_s) a.sig_s[gi] = (float)(1.0 / fmax(fmax(cx, cy), (cx + cy) / kSqrt2));
        if (a.tau_v) {
            a.tau_v[gi] = (float)(1.0 / (1 + 2 * A + kSqrt2 * B));
            a.tau_v[NN + gi] = (float)(1.0 / (1 + 2 * B + kSqrt2 * A));
        }
    }
}

__global__ void k_scale_f32(float* __restrict__ a, long long n, float m) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) a[i] *= m;
}

__global__ void k_sig_q(const float* __restrict__ krow, float* __restrict__ sig_q, long long S) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < S) {
        const double k = krow[i];
        sig_q[i] = k > 0 ? (float)(1.0 / k) : 1.f;
    }
}

// dst = src (N*N), or zero when src is NULL
__global__ void k_copy_or_zero(const float* __restrict__ src, float* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src ? src[i] : 0.f;
}

// Low words of a warm start, stored as the update stores them (bfloat16, see lo_encode).
__global__ void k_lo_encode(const float* __restrict__ lo, unsigned short* __restrict__ q, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        q[i] = lo_encode(lo[i]);
}

// Copies the final state out of the ping-pong buffers selected by the iteration count.
struct OutArgs {
    int n, reg;
    long long S;
    float theta;
    const float* X[2];
    const unsigned short* XL[2];   // low words of the compensated primal pairs (bfloat16)
    const float* Y[2];
    const float* q;
    const float* ubar;
    const InfoDev* info;
    float* u_out;
    float* x_out;
    float* x_lo_out;
    float* xbar_out;
    float* y_out;
};

__global__ void k_output(OutArgs a) {
    const int N = a.n;
    const long long NN = (long long)N * N;
    const int it = a.info->iter;
    const float* x = a.X[it & 1];
    const float* x_prev = a.X[(it + 1) & 1];
    const unsigned short* xl = a.XL[it & 1];
    const unsigned short* xl_prev = a.XL[(it + 1) & 1];
    const float* yrs = a.Y[(it + 1) & 1];  // r^I, s^I were read by the last update
    const int nv = a.reg == PAT_TGV ? 2 : 0;
    const long long nx = NN * (1 + nv), ny = NN * (a.reg == PAT_TGV ? 5 : 2);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nx + ny + a.S; i += stride) {
        if (i < nx) {
            if (i < NN && a.u_out) a.u_out[i] = x[i];
            if (a.x_out) a.x_out[i] = x[i];
            const float lo = lo_decode(xl[i]);
            if (a.x_lo_out) a.x_lo_out[i] = lo;
            if (a.xbar_out) {
                if (i < NN) {
                    a.xbar_out[i] = a.ubar[i];
                } else {
                    // vbar^I = v^I + theta (v^I - v^{I-1}) from the compensated pairs, the
                    // same expression as the update kernel's; with I = 0 the warm-start
                    // vbar is not recoverable here and v^0 is returned
                    const float lo_prev = lo_decode(xl_prev[i]);
                    a.xbar_out[i] = it > 0 ? fmaf(a.theta, (x[i] - x_prev[i]) + (lo - lo_prev), x[i] + lo)
                                           : x[i];
                }
            }
        } else if (a.y_out) {
            const long long j = i - nx;
            if (j < a.S)
                a.y_out[j] = a.q[j];
            else
                a.y_out[j] = yrs[j - a.S];
        }
    }
}

// ---------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
    float* X[2] = {nullptr, nullptr};
    unsigned short* XL[2] = {nullptr, nullptr};   // low words of the compensated primal pairs (bfloat16)
    float* Y[2] = {nullptr, nullptr};
    float *q = nullptr, *ubar = nullptr, *vbar0 = nullptr;
    int* kt[2] = {nullptr, nullptr};   // fixed-point K^T q, by iteration parity
    float *tau_u = nullptr, *sig_q = nullptr, *sig_r = nullptr, *qw = nullptr;
    double *data_part = nullptr, *pix_part = nullptr;
    InfoDev* info = nullptr;
    int n_data = 0, n_pix = 0;
};

static int pix_blocks(int N) { return std::min(4 * sm_count(), ceil_div((long long)N * N, 256)); }

static int alloc_workspace(const pat_geometry* g, int reg, Workspace& ws, cudaStream_t st) {
    const size_t N = g->desc.n, NN = N * N, S = (size_t)g->desc.n_det * g->desc.n_t;
    const size_t nx = NN * (reg == PAT_TGV ? 3 : 1), ny = NN * (reg == PAT_TGV ? 5 : 2);
    ws.n_data = g->fwd_n_ctas;   // one block of data-term sums per K CTA
    ws.n_pix = pix_blocks((int)N);
    size_t off[17];
    size_t sz[17] = {nx * 4, nx * 4, ny * 4, ny * 4, S * 4, NN * 4, NN * 4 * 2,
                     (reg == PAT_TGV ? 2 * NN : 1) * 4,
                     NN * 4, S * 4, NN * 4, (size_t)ws.n_data * GAP_DATA_TERMS * 8, (size_t)ws.n_pix * GAP_PIX_TERMS * 8, sizeof(InfoDev),
                     S * 4, nx * 2, nx * 2};
    size_t total = 0;
    for (int i = 0; i < 17; ++i) {
        off[i] = total;
        total += align_up(sz[i]);
    }
    PAT_CUDA(cudaMallocAsync(&ws.base, total, st));
    ws.bytes = total;
    char* b = (char*)ws.base;
    ws.X[0] = (float*)(b + off[0]);
    ws.X[1] = (float*)(b + off[1]);
    ws.Y[0] = (float*)(b + off[2]);
    ws.Y[1] = (float*)(b + off[3]);
    ws.q = (float*)(b + off[4]);
    ws.ubar = (float*)(b + off[5]);
    ws.kt[0] = (int*)(b + off[6]);
    ws.kt[1] = ws.kt[0] + NN;
    ws.vbar0 = (float*)(b + off[7]);
    ws.tau_u = (float*)(b + off[8]);
    ws.sig_q = (float*)(b + off[9]);
    ws.sig_r = (float*)(b + off[10]);
    ws.data_part = (double*)(b + off[11]);
    ws.pix_part = (double*)(b + off[12]);
    ws.info = (InfoDev*)(b + off[13]);
    ws.qw = (float*)(b + off[14]);
    ws.XL[0] = (unsigned short*)(b + off[15]);
    ws.XL[1] = (unsigned short*)(b + off[16]);
    return PAT_OK;
}

static int validate(const pat_geometry* g, const pat_params* p, const char* who) {
    char buf[256];
    auto bad = [&](const char* what) {
        snprintf(buf, sizeof buf, "%s: %s", who, what);
        return fail(PAT_ERR_INVALID_ARG, buf);
    };
    if (!g || !p) return bad("NULL geometry or params");
    if (p->reg < PAT_TV || p->reg > PAT_WAV) return bad("reg must be PAT_TV, PAT_TGV, PAT_DTV or PAT_WAV");
    if (p->reg == PAT_WAV) {
        const int J = p->wavelet_levels > 0 ? p->wavelet_levels : 4;
        if (!wav_levels_ok(g->desc.n, J)) return bad("PAT_WAV needs 1..12 levels and N divisible by 2^levels");
        if (p->precond != PAT_PRECOND_DIAG) return bad("PAT_WAV uses the diagonal steps only");
        if (p->adapt != PAT_ADAPT_NONE) return bad("PAT_WAV has no adaptive balance");
        if (p->wavelet_kind != PAT_WAVELET_DWT && p->wavelet_kind != PAT_WAVELET_DTCWT)
            return bad("wavelet_kind must be PAT_WAVELET_DWT or PAT_WAVELET_DTCWT");
        if (p->wavelet_kind == PAT_WAVELET_DTCWT) {
            CwtBank bank;
            const int frc = cwt_bank(p->dtcwt_h1_host, p->dtcwt_l1, p->dtcwt_hq_host, p->dtcwt_lq, bank, nullptr, nullptr);
            if (frc) return frc;
        }
    }
    if (!(p->alpha >= 0) || !std::isfinite(p->alpha)) return bad("alpha must be finite and >= 0");
    if (!(p->beta >= 0) || !std::isfinite(p->beta)) return bad("beta must be finite and >= 0");
    if (p->reg == PAT_DTV && (!(p->gamma >= 0) || !(p->gamma <= 1))) return bad("gamma must be in [0, 1]");
    if (p->reg == PAT_DTV && !p->xi_dev) return bad("directional TV needs xi_dev");
    if (p->iters < 0) return bad("iters must be >= 0");
    if (!(p->tol >= 0)) return bad("tol must be >= 0");
    if (p->gap_every < 0) return bad("gap_every must be >= 0");
    if (p->precond != PAT_PRECOND_DIAG && p->precond != PAT_PRECOND_SCALAR2) return bad("unknown precond");
    if (!(p->theta >= 0) || !(p->theta <= 1)) return bad("theta must be in [0, 1]");
    if (!(p->box_u > 0) || !(p->box_v > 0)) return bad("box half-widths must be > 0");
    if (!(p->step_ratio >= 0) || !std::isfinite(p->step_ratio)) return bad("step_ratio must be finite and >= 0");
    if (p->adapt != PAT_ADAPT_NONE && p->adapt != PAT_ADAPT_BALANCE) return bad("unknown adapt mode");
    return PAT_OK;
}

// s of the primal-dual balance; 0 (a zero-initialised struct) means the default 1.
static double step_ratio_of(const pat_params* p) { return p->step_ratio > 0 ? p->step_ratio : 1.0; }

struct ScalarSteps {
    float sig_q = -1.f, sig2 = -1.f, tau = -1.f;
};

int scalar2_steps(const pat_geometry* g, const pat_params* p, ScalarSteps& out, cudaStream_t st);

// Fills the step arrays in ws (diagonal rule) or the scalars (paper rule).
static int compute_steps(const pat_geometry* g, const pat_params* p, Workspace& ws, ScalarSteps& sc,
                         cudaStream_t st) {
    const int N = g->desc.n;
    const long long S = (long long)g->desc.n_det * g->desc.n_t;
    int rc = ensure_precond(g, st);  // K sums also scale the fixed-point K^T
    if (rc) return rc;
    if (p->precond == PAT_PRECOND_SCALAR2) return scalar2_steps(g, p, sc, st);
    k_sig_q<<<ceil_div(S, 256), 256, 0, st>>>(g->pc.krow, ws.sig_q, S);
    PAT_LAUNCH_CHECK("k_sig_q");
    StepArgs sa{N, p->reg, p->gamma, g->pc.kcol, p->xi_dev, ws.tau_u, p->reg == PAT_DTV ? ws.sig_r : nullptr,
                nullptr, nullptr};
    dim3 blk(32, 8), grd(ceil_div(N, 32), ceil_div(N, 8));
    k_steps_pixels<<<grd, blk, 0, st>>>(sa);
    PAT_LAUNCH_CHECK("k_steps_pixels");
    return PAT_OK;
}

// ---------------------------------------------------------------------------------
// batch engine: problems advance in lockstep; one launch per phase covers all of them
// through a (problem, local block) map, and the periodic part of the iteration loop is
// replayed from a captured CUDA graph.  A single reconstruction is a batch of one.
// ---------------------------------------------------------------------------------
struct Prob {
    const pat_geometry* g = nullptr;
    const float* f = nullptr;
    pat_params p{};
    float* u_out = nullptr;
    Workspace ws;
    ScalarSteps sc;
};

// Packs host-side argument structs and maps, then uploads them in one copy.
struct Arena {
    std::vector<char>& buf;
    explicit Arena(std::vector<char>& b) : buf(b) {}
    template <class T>
    size_t put(const T* p, size_t n) {
        const size_t off = align_up(buf.size());
        buf.resize(off + std::max<size_t>(1, n) * sizeof(T));
        if (n) memcpy(buf.data() + off, p, n * sizeof(T));
        return off;
    }
    int upload(void** dev, cudaStream_t st) {
        PAT_CUDA(cudaMallocAsync(dev, buf.size(), st));
        PAT_CUDA(cudaMemcpyAsync(*dev, buf.data(), buf.size(), cudaMemcpyHostToDevice, st));
        return PAT_OK;
    }
};

// K launches of a batch: problems with the same cluster size (slabs) share a launch
struct FwdGroup {
    int cluster = 1, smem = 0, n = 0;   // CTAs per cluster, dynamic shared memory, CTAs
    size_t map = 0;                     // (problem, CTA) pairs, cluster-major, rank-minor
};

struct GapPlan {
    FwdGroup fwd[FWD_MAX_CLUSTER];
    int n_fwd_groups = 0;
    size_t map_pix[3] = {0, 0, 0};
    int n_pix[3] = {0, 0, 0};
};

// The K launch groups of a batch.  In each, clusters run longest first: their work differs
// and a launch may span several waves, so the order sets the length of the last wave (each
// cluster's rows do not depend on it).
static void forward_groups(const Prob* pr, int B, Arena& ar, GapPlan& gp) {
    gp.n_fwd_groups = 0;
    for (int S = 1; S <= FWD_MAX_CLUSTER; ++S) {
        std::vector<std::pair<float, int2>> v;   // (cost, (problem, cluster))
        int smem = 0;
        for (int b = 0; b < B; ++b) {
            const pat_geometry* g = pr[b].g;
            if (g->view.n_slabs != S) continue;
            smem = std::max(smem, g->fwd_smem);
            for (int c = 0; c < (int)g->fwd_cluster_cost.size(); ++c) v.push_back({g->fwd_cluster_cost[c], make_int2(b, c)});
        }
        if (v.empty()) continue;
        std::stable_sort(v.begin(), v.end(), [](const std::pair<float, int2>& x, const std::pair<float, int2>& y) {
            return x.first > y.first;
        });
        std::vector<int2> m;
        m.reserve(v.size() * S);
        for (auto& e : v)
            for (int r = 0; r < S; ++r) m.push_back(make_int2(e.second.x, e.second.y * S + r));
        FwdGroup& grp = gp.fwd[gp.n_fwd_groups++];
        grp.cluster = S;
        grp.smem = smem;
        grp.n = (int)m.size();
        grp.map = ar.put(m.data(), m.size());
    }
}

static int launch_forward_groups(int epi, const FwdArgs* args, const GapPlan& gp, const char* base, cudaStream_t st) {
    for (int i = 0; i < gp.n_fwd_groups; ++i) {
        const FwdGroup& grp = gp.fwd[i];
        const int rc = launch_forward_b(epi, args, (const int2*)(base + grp.map), grp.n, grp.cluster, grp.smem, st);
        if (rc) return rc;
    }
    return PAT_OK;
}

static void build_gap_plan(const Prob* pr, int B, Arena& ar, GapPlan& gp) {
    std::vector<int2> pix[3];
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < pr[b].ws.n_pix; ++i) pix[pr[b].p.reg].push_back(make_int2(b, i));
    forward_groups(pr, B, ar, gp);
    for (int r = 0; r < 3; ++r) {
        gp.map_pix[r] = ar.put(pix[r].data(), pix[r].size());
        gp.n_pix[r] = (int)pix[r].size();
    }
}

static GapArgs make_gap_args(const Prob& pr, const KtView& kt, const float* x, const float* x_old, const float* y_rs) {
    GapArgs ga;
    ga.n = pr.g->desc.n;
    ga.alpha = (float)pr.p.alpha;
    ga.ab = (float)(pr.p.alpha * pr.p.beta);
    ga.gamma = pr.p.gamma;
    ga.xi = pr.p.xi_dev;
    ga.x = x;
    ga.x_old = x_old;
    ga.y = y_rs;
    ga.kt = kt;
    ga.partials = pr.ws.pix_part;
    ga.stop = &pr.ws.info->stop;
    ga.nblocks = pr.ws.n_pix;
    return ga;
}

static FinalArgs make_final_args(const Prob& pr, int* batch_stopped = nullptr) {
    FinalArgs fa{pr.ws.data_part, pr.ws.n_data, pr.ws.pix_part, pr.ws.n_pix, pr.p.alpha, pr.p.beta, pr.p.box_u,
                 pr.p.box_v, pr.p.tol, pr.p.reg, pr.p.adapt, pr.ws.info, batch_stopped};
    return fa;
}

static UpdateArgs make_update_args(const Prob& pr, int par, bool gap_iter) {
    const Workspace& ws = pr.ws;
    const pat_params* p = &pr.p;
    const int N = pr.g->desc.n;
    UpdateArgs a;
    a.n = N;
    a.alpha = (float)p->alpha;
    a.ab = (float)(p->alpha * p->beta);
    a.gamma = (float)p->gamma;
    a.theta = (float)p->theta;
    a.sig2 = pr.sc.sig2;
    a.tau = pr.sc.tau;
    a.tau_u = ws.tau_u;
    a.sig_r = ws.sig_r;
    a.xi = p->xi_dev;
    a.step_mul = ws.info->step_mul;
    a.kt = kt_view(pr.g, ws.kt[par], &ws.info->qmax_bits[par]);
    a.kt_clear = ws.kt[1 - par];
    a.qmax_next = &ws.info->qmax_bits[1 - par];
    a.x_in = ws.X[par];
    a.xl_in = ws.XL[par];
    a.y_in = ws.Y[par];
    a.x_out = ws.X[1 - par];
    a.xl_out = ws.XL[1 - par];
    a.y_out = ws.Y[1 - par];
    a.ubar = ws.ubar;
    (void)gap_iter;
    a.stop = &ws.info->stop;
    a.iter = &ws.info->iter;
    a.tiles_x = ceil_div(N, upd_tx(pr.g->shapes.update_tile));
    return a;
}

template <int TILE>
static void launch_update_tile(int reg, const UpdateArgs* args, const int2* map, int n, cudaStream_t st) {
    const dim3 blk(upd_tx(TILE), upd_ty(TILE));
    if (reg == PAT_TV)
        k_update_b<PAT_TV, TILE><<<n, blk, 0, st>>>(args, map);
    else if (reg == PAT_TGV)
        k_update_b<PAT_TGV, TILE><<<n, blk, 0, st>>>(args, map);
    else
        k_update_b<PAT_DTV, TILE><<<n, blk, 0, st>>>(args, map);
}

static int launch_update_b(int reg, int tile, const UpdateArgs* args, const int2* map, int n, cudaStream_t st) {
    if (n <= 0) return PAT_OK;
    prof_mark(PAT_PHASE_UPDATE, st, true);
    if (tile == PAT_UPD_64X4)
        launch_update_tile<PAT_UPD_64X4>(reg, args, map, n, st);
    else if (tile == PAT_UPD_32X8)
        launch_update_tile<PAT_UPD_32X8>(reg, args, map, n, st);
    else
        launch_update_tile<PAT_UPD_32X4>(reg, args, map, n, st);
    PAT_LAUNCH_CHECK("k_update_b");
    prof_mark(PAT_PHASE_UPDATE, st, false);
    return PAT_OK;
}

static int launch_gap_phase(const FwdArgs* fa, const GapArgs* ga, const FinalArgs* fi, const GapPlan& gp,
                            const char* base, cudaStream_t st) {
    prof_mark(PAT_PHASE_GAP, st, true);
    int rc = launch_forward_groups(FWD_GAP, fa, gp, base, st);
    if (rc) return rc;
    for (int r = 0; r < 3; ++r) {
        if (!gp.n_pix[r]) continue;
        const int2* map = (const int2*)(base + gp.map_pix[r]);
        if (r == PAT_TV)
            k_gap_pixels_final_b<PAT_TV><<<gp.n_pix[r], 256, 0, st>>>(ga, fi, map);
        else if (r == PAT_TGV)
            k_gap_pixels_final_b<PAT_TGV><<<gp.n_pix[r], 256, 0, st>>>(ga, fi, map);
        else
            k_gap_pixels_final_b<PAT_DTV><<<gp.n_pix[r], 256, 0, st>>>(ga, fi, map);
        PAT_LAUNCH_CHECK("k_gap_pixels_final_b");
    }
    prof_mark(PAT_PHASE_GAP, st, false);
    return PAT_OK;
}

struct IterPlan {
    size_t fwd[2] = {0, 0}, adj[2] = {0, 0}, upd[2][2] = {{0, 0}, {0, 0}}, fgap[2] = {0, 0}, gpix[2] = {0, 0};
    size_t fin = 0, map_adj = 0;
    size_t map_upd[3][UPD_TILES] = {};
    int n_adj = 0;
    int n_upd[3][UPD_TILES] = {};
    GapPlan gp;
};

static void build_iter_plan(const Prob* pr, int B, Arena& ar, IterPlan& ip, int* batch_stopped) {
    for (int par = 0; par < 2; ++par) {
        std::vector<FwdArgs> fw;
        std::vector<AdjArgs> ad;
        std::vector<UpdateArgs> u0, u1;
        std::vector<FwdArgs> fg;
        std::vector<GapArgs> gpx;
        for (int b = 0; b < B; ++b) {
            const Prob& q = pr[b];
            const Workspace& ws = q.ws;
            FwdArgs fa = make_fwd_args(q.g, ws.ubar);
            fa.q = ws.q;
            fa.f = q.f;
            fa.sig_q = q.sc.sig_q >= 0 ? nullptr : ws.sig_q;
            fa.sig_scalar = q.sc.sig_q;
            fa.step_mul = ws.info->step_mul;
            fa.qw = ws.qw;
            fa.qmax_bits = &ws.info->qmax_bits[par];
            fa.stop = &ws.info->stop;
            fw.push_back(fa);
            ad.push_back(make_adj_args(q.g, ws.q, ws.qw, &ws.info->qmax_bits[par], ws.kt[par], &ws.info->stop));
            u0.push_back(make_update_args(q, par, false));
            u1.push_back(make_update_args(q, par, true));
            // the gap's K u reads the high words of u^{n+1}, the FP32 value of the pair
            FwdArgs ga = make_fwd_args(q.g, ws.X[1 - par]);
            ga.q = ws.q;
            ga.f = q.f;
            ga.partials = ws.data_part;
            ga.stop = &ws.info->stop;
            fg.push_back(ga);
            gpx.push_back(make_gap_args(q, kt_view(q.g, ws.kt[par], &ws.info->qmax_bits[par]), ws.X[1 - par],
                                        ws.X[par], ws.Y[par]));
        }
        ip.fwd[par] = ar.put(fw.data(), fw.size());
        ip.adj[par] = ar.put(ad.data(), ad.size());
        ip.upd[par][0] = ar.put(u0.data(), u0.size());
        ip.upd[par][1] = ar.put(u1.data(), u1.size());
        ip.fgap[par] = ar.put(fg.data(), fg.size());
        ip.gpix[par] = ar.put(gpx.data(), gpx.size());
    }
    std::vector<FinalArgs> fi;
    for (int b = 0; b < B; ++b) fi.push_back(make_final_args(pr[b], batch_stopped));
    ip.fin = ar.put(fi.data(), fi.size());
    // maps: forward rows problem by problem; K^T items of all problems heaviest first;
    // update tiles grouped by regulariser
    std::vector<int2> upd[3][UPD_TILES];
    std::vector<std::pair<float, int2>> adj;
    for (int b = 0; b < B; ++b) {
        const pat_geometry* g = pr[b].g;
        for (int i = 0; i < g->adj_items; ++i) adj.push_back({g->adj_item_cost[i], make_int2(b, i)});
        const int tile = g->shapes.update_tile;
        const int N = g->desc.n, nt = ceil_div(N, upd_tx(tile)) * ceil_div(N, upd_ty(tile));
        for (int i = 0; i < nt; ++i) upd[pr[b].p.reg][tile].push_back(make_int2(b, i));
    }
    std::stable_sort(adj.begin(), adj.end(), [](const std::pair<float, int2>& x, const std::pair<float, int2>& y) {
        return x.first > y.first;
    });
    std::vector<int2> adjm;
    for (auto& e : adj) adjm.push_back(e.second);
    ip.map_adj = ar.put(adjm.data(), adjm.size());
    ip.n_adj = (int)adjm.size();
    for (int r = 0; r < 3; ++r)
        for (int t = 0; t < UPD_TILES; ++t) {
            ip.map_upd[r][t] = ar.put(upd[r][t].data(), upd[r][t].size());
            ip.n_upd[r][t] = (int)upd[r][t].size();
        }
    build_gap_plan(pr, B, ar, ip.gp);
}

static int enqueue_iteration(const IterPlan& ip, const char* base, int it, bool gap_due, cudaStream_t st) {
    const int par = it & 1;
    int rc = launch_forward_groups(FWD_PROX, (const FwdArgs*)(base + ip.fwd[par]), ip.gp, base, st);
    if (rc) return rc;
    rc = launch_adjoint_b((const AdjArgs*)(base + ip.adj[par]), (const int2*)(base + ip.map_adj), ip.n_adj, true, st);
    if (rc) return rc;
    const UpdateArgs* ua = (const UpdateArgs*)(base + ip.upd[par][gap_due ? 1 : 0]);
    for (int r = 0; r < 3; ++r)
        for (int t = 0; t < UPD_TILES; ++t) {
            rc = launch_update_b(r, t, ua, (const int2*)(base + ip.map_upd[r][t]), ip.n_upd[r][t], st);
            if (rc) return rc;
        }
    if (gap_due)
        rc = launch_gap_phase((const FwdArgs*)(base + ip.fgap[par]), (const GapArgs*)(base + ip.gpix[par]),
                              (const FinalArgs*)(base + ip.fin), ip.gp, base, st);
    return rc;
}

// initial state of one problem (Algorithm 1/2 initialisation, or the warm start)
static int init_problem(Prob& pr, cudaStream_t st) {
    const pat_geometry* g = pr.g;
    const pat_params* p = &pr.p;
    const int reg = p->reg;
    const int N = g->desc.n;
    const size_t NN = (size_t)N * N, S = (size_t)g->desc.n_det * g->desc.n_t;
    const size_t nx = NN * (reg == PAT_TGV ? 3 : 1), ny = NN * (reg == PAT_TGV ? 5 : 2);
    Workspace& ws = pr.ws;
    int rc = alloc_workspace(g, reg, ws, st);
    if (rc) return rc;
    rc = compute_steps(g, p, ws, pr.sc, st);
    if (rc) return rc;
    if (p->x0_dev)
        PAT_CUDA(cudaMemcpyAsync(ws.X[0], p->x0_dev, nx * 4, cudaMemcpyDeviceToDevice, st));
    else
        PAT_CUDA(cudaMemsetAsync(ws.X[0], 0, nx * 4, st));
    if (p->y0_dev) {
        PAT_CUDA(cudaMemcpyAsync(ws.q, p->y0_dev, S * 4, cudaMemcpyDeviceToDevice, st));
        PAT_CUDA(cudaMemcpyAsync(ws.Y[1], p->y0_dev + S, ny * 4, cudaMemcpyDeviceToDevice, st));
    } else {
        PAT_CUDA(cudaMemsetAsync(ws.q, 0, S * 4, st));
        PAT_CUDA(cudaMemsetAsync(ws.Y[1], 0, ny * 4, st));
    }
    PAT_CUDA(cudaMemsetAsync(ws.info, 0, sizeof(InfoDev), st));
    const double ratio = step_ratio_of(p);
    const float mul[2] = {(float)ratio, (float)(1.0 / ratio)};
    PAT_CUDA(cudaMemcpyAsync(ws.info->step_mul, mul, sizeof mul, cudaMemcpyHostToDevice, st));
    PAT_CUDA(cudaMemsetAsync(ws.kt[0], 0, 2 * NN * sizeof(int), st));
    if (p->x_lo0_dev) {
        k_lo_encode<<<std::min(4 * sm_count(), ceil_div((long long)nx, 256)), 256, 0, st>>>(p->x_lo0_dev, ws.XL[0],
                                                                                            (long long)nx);
        PAT_LAUNCH_CHECK("k_lo_encode");
    } else {
        PAT_CUDA(cudaMemsetAsync(ws.XL[0], 0, nx * sizeof(unsigned short), st));
    }
    const float* xb = p->xbar0_dev ? p->xbar0_dev : p->x0_dev;
    k_copy_or_zero<<<std::min(4 * sm_count(), ceil_div((long long)NN, 256)), 256, 0, st>>>(xb, ws.ubar, (long long)NN);
    PAT_LAUNCH_CHECK("k_copy_or_zero");
    if (reg == PAT_TGV) {
        if (xb)
            PAT_CUDA(cudaMemcpyAsync(ws.vbar0, xb + NN, 2 * NN * 4, cudaMemcpyDeviceToDevice, st));
        else
            PAT_CUDA(cudaMemsetAsync(ws.vbar0, 0, 2 * NN * 4, st));
    }
    // dual prologue: (r^1, s^1) from (r^0, s^0) and (ubar^0, vbar^0) into Y[0]
    DualArgs da{N, (float)p->alpha, (float)(p->alpha * p->beta), (float)p->gamma, pr.sc.sig2, mul[1], ws.sig_r,
                p->xi_dev, ws.ubar, ws.vbar0, ws.Y[1], ws.Y[0]};
    dim3 blk(32, 8), g2(ceil_div(N, 32), ceil_div(N, 8));
    if (reg == PAT_TV)
        k_dual_step<PAT_TV><<<g2, blk, 0, st>>>(da);
    else if (reg == PAT_TGV)
        k_dual_step<PAT_TGV><<<g2, blk, 0, st>>>(da);
    else
        k_dual_step<PAT_DTV><<<g2, blk, 0, st>>>(da);
    PAT_LAUNCH_CHECK("k_dual_step");
    return PAT_OK;
}

static int finish_problem(Prob& pr, cudaStream_t st) {
    const pat_geometry* g = pr.g;
    const int reg = pr.p.reg;
    const int N = g->desc.n;
    const size_t NN = (size_t)N * N, S = (size_t)g->desc.n_det * g->desc.n_t;
    const size_t nx = NN * (reg == PAT_TGV ? 3 : 1), ny = NN * (reg == PAT_TGV ? 5 : 2);
    OutArgs oa;
    oa.n = N;
    oa.reg = reg;
    oa.S = (long long)S;
    oa.theta = (float)pr.p.theta;
    oa.X[0] = pr.ws.X[0];
    oa.X[1] = pr.ws.X[1];
    oa.XL[0] = pr.ws.XL[0];
    oa.XL[1] = pr.ws.XL[1];
    oa.Y[0] = pr.ws.Y[0];
    oa.Y[1] = pr.ws.Y[1];
    oa.q = pr.ws.q;
    oa.ubar = pr.ws.ubar;
    oa.info = pr.ws.info;
    oa.u_out = pr.u_out;
    oa.x_out = pr.p.x_out_dev;
    oa.x_lo_out = pr.p.x_lo_out_dev;
    oa.xbar_out = pr.p.xbar_out_dev;
    oa.y_out = pr.p.y_out_dev;
    k_output<<<std::min(2 * sm_count(), ceil_div((long long)(nx + ny + S), 256)), 256, 0, st>>>(oa);
    PAT_LAUNCH_CHECK("k_output");
    return PAT_OK;
}

// A non-blocking stream per device for the iteration loop (capturable, unlike the legacy
// default stream); it is joined to the caller's stream with events.
static cudaStream_t loop_stream() {
    static thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

// Pinned host slots for the stop-counter snapshots of run_iterations (one pair per thread).
static int* stop_snapshots() {
    thread_local int* h = nullptr;
    if (!h && cudaHostAlloc((void**)&h, 2 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        h = nullptr;
    }
    return h;
}

// Enqueues all iterations.  The periodic part replays a captured graph in chunks of
// CHUNK periods.  When the batch can stop early (some problem has a tolerance), the
// counter of stopped problems is copied to pinned memory after every chunk.  Before the
// next chunk is enqueued, the host reads the previous chunk's copy; the GPU is then busy
// with the current chunk, so it never idles.  Replays end once every problem has stopped:
// the kernels of a stopped problem return at entry, but their launches still cost time.
static int run_iterations(const IterPlan& ip, const char* base, int iters, int ge, cudaStream_t st,
                          const int* batch_stopped, int B, bool can_stop) {
    auto gap_due = [&](int it) { return (ge > 0 && (it + 1) % ge == 0) || it + 1 == iters; };
    const int P = ge > 0 ? (ge % 2 == 0 ? ge : 2 * ge) : 2;
    const int nper = iters > 0 ? (iters - 1) / P : 0;
    int start = 0;
    bool all_stopped = false;
    if (!prof_on() && nper >= 2) {
        // one period of the loop as a graph; periods repeat exactly (P is even, so the
        // ping-pong parity repeats, and a multiple of gap_every, so the gap passes do)
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const long long l0 = pat_kernel_launches();
        PAT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = PAT_OK;
        for (int it = 0; it < P && !rc; ++it) rc = enqueue_iteration(ip, base, it, ge > 0 && (it + 1) % ge == 0, st);
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "run_iterations: graph capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(e, "run_iterations: graph instantiate");
        }
        const long long per_period = pat_kernel_launches() - l0;
        constexpr int CHUNK = 8;
        int* snap = can_stop && batch_stopped ? stop_snapshots() : nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        bool pending[2] = {false, false};
        if (snap)
            for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        int launched = 0;
        for (int chunk = 0; launched < nper && e == cudaSuccess; ++chunk) {
            const int n = std::min(CHUNK, nper - launched);
            for (int r = 0; r < n && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, st);
            launched += n;
            if (!snap || e != cudaSuccess) continue;
            const int cur = chunk & 1, prev = cur ^ 1;
            e = cudaMemcpyAsync(&snap[cur], batch_stopped, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(ev[cur], st);
            pending[cur] = e == cudaSuccess;
            if (pending[prev] && e == cudaSuccess) {
                e = cudaEventSynchronize(ev[prev]);
                pending[prev] = false;
                if (e == cudaSuccess && *(volatile int*)&snap[prev] >= B) {
                    all_stopped = true;
                    break;
                }
            }
        }
        for (int i = 0; i < 2; ++i)
            if (ev[i]) {
                if (pending[i]) cudaEventSynchronize(ev[i]);   // the slot is reused by the next call
                cudaEventDestroy(ev[i]);
            }
        for (int r = 1; r < launched; ++r)
            for (long long k = 0; k < per_period; ++k) count_launch();
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "run_iterations: graph launch");
        start = nper * P;
    }
    if (all_stopped) return PAT_OK;
    for (int it = start; it < iters; ++it) {
        int rc = enqueue_iteration(ip, base, it, gap_due(it), st);
        if (rc) return rc;
    }
    return PAT_OK;
}

// ---------------------------------------------------------------------------------
// the wavelet model (Sec. 2.2 eq. (min_wav)): Algorithm 1 with grad -> W and div -> -W^T
// (Sec. 3.3).  One problem at a time; the periodic part of the loop is a captured graph
// like the batch engine's, and it ends early once the problem has stopped.
//   q^{n+1} = prox(q^n + S K ubar^n),  r^{n+1} = clip(r^n + S_r W ubar^n, alpha),
//   u^{n+1} = u^n - T (K^T q^{n+1} + W^T r^{n+1}),  ubar^{n+1} = u^{n+1} + theta (u^{n+1} - u^n)
// ---------------------------------------------------------------------------------
static int wav_levels_of(const pat_params* p) { return p->wavelet_levels > 0 ? p->wavelet_levels : 4; }

// The transform of a PAT_WAV problem: the orthonormal DWT (N^2 coefficients) or the
// DT-CWT (4 N^2 coefficients, four planes) with its filter bank.
struct WavModel {
    int kind = PAT_WAVELET_DWT, J = 4, N = 0;
    long long nr = 0;
    CwtBank bank{};
    std::vector<double> h1, hq;
    // the |W| row sums (with the DT-CWT, paired per complex coefficient) and column sums,
    // filled by the first wav_steps call and shared by the problems of a batch
    std::vector<double> rows, cols;
};

static int wav_model(const pat_geometry* g, const pat_params* p, WavModel& m) {
    m.kind = p->wavelet_kind;
    m.J = wav_levels_of(p);
    m.N = g->desc.n;
    const long long NN = (long long)m.N * m.N;
    m.nr = m.kind == PAT_WAVELET_DTCWT ? 4 * NN : NN;
    if (m.kind == PAT_WAVELET_DTCWT)
        return cwt_bank(p->dtcwt_h1_host, p->dtcwt_l1, p->dtcwt_hq_host, p->dtcwt_lq, m.bank, &m.h1, &m.hq);
    return PAT_OK;
}

// Two wavelet problems can share a batch when they have one N and one transform (kind,
// levels and, for the DT-CWT, filters)
static bool wav_same_batch(const pat_geometry* ga, const pat_params* pa, const pat_geometry* gb, const pat_params* pb) {
    if (ga->desc.n != gb->desc.n || wav_levels_of(pa) != wav_levels_of(pb) || pa->wavelet_kind != pb->wavelet_kind)
        return false;
    if (pa->wavelet_kind != PAT_WAVELET_DTCWT) return true;
    WavModel ma, mb;
    if (wav_model(ga, pa, ma) || wav_model(gb, pb, mb)) return false;
    return ma.h1 == mb.h1 && ma.hq == mb.hq;
}

// sigma_q, tau_u and sigma_r of the wavelet model: the alpha = 1 diagonal rule on A = (K; W).
// With the DT-CWT the two rows of a complex coefficient share one step, 1 / (the larger of
// their row sums): the dual prox of a disc is the projection onto it only with one step.
static int wav_steps(const pat_geometry* g, WavModel& m, float* sig_q, float* tau_u, float* sig_r,
                     double s_ratio, cudaStream_t st) {
    const int N = g->desc.n;
    const long long NN = (long long)N * N, S = (long long)g->desc.n_det * g->desc.n_t;
    int rc = ensure_precond(g, st);
    if (rc) return rc;
    std::vector<double>& rows = m.rows;
    std::vector<double>& cols = m.cols;
    if (rows.empty() && m.kind == PAT_WAVELET_DTCWT) {
        cwt_abs_sums(N, m.J, m.h1, m.hq, rows, cols);
        const int side = N >> m.J;
        for (long long i = 0; i < NN; ++i) {
            if ((int)(i % N) < side && (int)(i / N) < side) continue;   // LL: one row each
            for (int a = 0; a < 4; a += 2) {
                const double mx = std::max(rows[a * NN + i], rows[(a + 1) * NN + i]);
                rows[a * NN + i] = rows[(a + 1) * NN + i] = mx;
            }
        }
    } else if (rows.empty()) {
        wav_abs_sums(N, m.J, rows, cols);
    }
    if (sig_q) {
        k_sig_q<<<ceil_div(S, 256), 256, 0, st>>>(g->pc.krow, sig_q, S);
        PAT_LAUNCH_CHECK("k_sig_q");
        if (s_ratio != 1.0) {
            k_scale_f32<<<ceil_div(S, 256), 256, 0, st>>>(sig_q, S, (float)(1.0 / s_ratio));
            PAT_LAUNCH_CHECK("k_scale_f32");
        }
    }
    if (tau_u) {
        double* wcol = nullptr;
        PAT_CUDA(cudaMallocAsync(&wcol, NN * sizeof(double), st));
        rc = cudaMemcpyAsync(wcol, cols.data(), NN * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess
                 ? launch_wav_tau(g->pc.kcol, wcol, tau_u, NN, st)
                 : fail(PAT_ERR_CUDA, "wav_steps: copy");
        if (!rc) PAT_CUDA(cudaStreamSynchronize(st));   // the host vector dies with this call
        cudaFreeAsync(wcol, st);
        if (rc) return rc;
        if (s_ratio != 1.0) {
            k_scale_f32<<<ceil_div(NN, 256), 256, 0, st>>>(tau_u, NN, (float)s_ratio);
            PAT_LAUNCH_CHECK("k_scale_f32");
        }
    }
    if (sig_r) {
        std::vector<float> h((size_t)m.nr);
        for (long long i = 0; i < m.nr; ++i) h[i] = rows[i] > 0 ? (float)(1.0 / rows[i] / s_ratio) : 1.f;
        PAT_CUDA(cudaMemcpyAsync(sig_r, h.data(), m.nr * sizeof(float), cudaMemcpyHostToDevice, st));
        PAT_CUDA(cudaStreamSynchronize(st));
    }
    return PAT_OK;
}

// B problems of the wavelet model that share N, the transform with its levels and filters,
// the iteration count and the gap period advance in lockstep, as in the batch engine: K and
// K^T launch once for all problems through (problem, block) maps (clusters and work items
// of all problems heaviest first), and every wavelet kernel covers all problems through a
// problem index in its grid, each problem's buffers in one workspace block at a fixed byte
// stride.  A single reconstruction is a batch of one.
static int run_wavelet(int B, const pat_geometry* const* g, const float* const* f, const pat_params* p,
                       float* const* u_out, pat_info* infos, cudaStream_t st, const char* who) {
    if (B <= 0) return PAT_OK;
    const int N = g[0]->desc.n, J = wav_levels_of(&p[0]);
    const long long NN = (long long)N * N;
    const int n_pix = pix_blocks(N);
    WavModel wm;
    if (int mrc = wav_model(g[0], &p[0], wm)) return mrc;
    const bool cwt = wm.kind == PAT_WAVELET_DTCWT;
    const long long NR = wm.nr;   // coefficients of W u
    long long S = 0;              // the largest data size and K CTA count of the batch
    int n_data = 0;
    for (int b = 0; b < B; ++b) {
        if (g[b]->desc.n != N) return fail(PAT_ERR_INVALID_ARG, std::string(who) + ": a wavelet batch needs one N");
        S = std::max(S, (long long)g[b]->desc.n_det * g[b]->desc.n_t);
        n_data = std::max(n_data, g[b]->fwd_n_ctas);
    }
    // one workspace block per problem (DT-CWT: R, WB, WU and SIGR hold 4 planes, SCRT the
    // tree form of r); SCAL holds {alpha, theta}, TKM the geometry's K^T tile bounds
    enum { U, UOLD, UBAR, Q, QW, KT, R, WB, WTR, SCR, SCR2, WU, TAU, SIGR, SIGQ, DPART, PPART, INFO, SCRT, SCAL, TKM,
           NBUF };
    // SCR, SCR2: transform scratch (DT-CWT: the LL blocks passed between levels, 5 N^2 / 4)
    const size_t nn4 = (size_t)NN * 4, nr4 = (size_t)NR * 4, scr4 = cwt ? nn4 + nn4 / 4 : nn4;
    const size_t sz[NBUF] = {nn4, nn4, nn4, (size_t)S * 4, (size_t)S * 4, (size_t)NN * 8, nr4, nr4, nn4, scr4, scr4,
                             nr4, nn4, nr4, (size_t)S * 4, (size_t)n_data * GAP_DATA_TERMS * 8,
                             (size_t)n_pix * GAP_PIX_TERMS * 8, sizeof(InfoDev), cwt ? nr4 : 16, 2 * sizeof(float),
                             (size_t)g[0]->adj_tiles * sizeof(float)};
    size_t off[NBUF], PS = 0;
    for (int i = 0; i < NBUF; ++i) {
        off[i] = PS;
        PS += align_up(sz[i]);
    }
    const long long ps = (long long)PS;
    char* ws = nullptr;
    PAT_CUDA(cudaMallocAsync((void**)&ws, PS * (size_t)B, st));
    auto buf = [&](int b, int i) { return ws + (size_t)b * PS + off[i]; };
    auto F = [&](int b, int i) { return (float*)buf(b, i); };
    auto inf = [&](int b) { return (InfoDev*)buf(b, INFO); };
    cudaEvent_t e0, e1;
    PAT_CUDA(cudaEventCreate(&e0));
    PAT_CUDA(cudaEventCreate(&e1));
    PAT_CUDA(cudaEventRecord(e0, st));
    int rc = PAT_OK;
    auto cp = [&](float* dst, const float* src, long long n) -> int {
        if (src) PAT_CUDA(cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, st));
        else PAT_CUDA(cudaMemsetAsync(dst, 0, n * 4, st));
        return PAT_OK;
    };
    for (int b = 0; b < B && !rc; ++b) {
        const long long Sb = (long long)g[b]->desc.n_det * g[b]->desc.n_t;
        rc = wav_steps(g[b], wm, F(b, SIGQ), F(b, TAU), F(b, SIGR), 1.0, st);
        if (!rc) rc = cp(F(b, U), p[b].x0_dev, NN);
        if (!rc) rc = cp(F(b, UBAR), p[b].xbar0_dev ? p[b].xbar0_dev : p[b].x0_dev, NN);
        if (!rc) rc = cp(F(b, Q), p[b].y0_dev, Sb);
        if (!rc) rc = cp(F(b, R), p[b].y0_dev ? p[b].y0_dev + Sb : nullptr, NR);
        if (rc) break;
        PAT_CUDA(cudaMemsetAsync(inf(b), 0, sizeof(InfoDev), st));
        const double ratio = step_ratio_of(&p[b]);
        const float mul[2] = {(float)ratio, (float)(1.0 / ratio)};
        PAT_CUDA(cudaMemcpyAsync(inf(b)->step_mul, mul, sizeof mul, cudaMemcpyHostToDevice, st));
        const float scal[2] = {(float)p[b].alpha, (float)p[b].theta};
        PAT_CUDA(cudaMemcpyAsync(F(b, SCAL), scal, sizeof scal, cudaMemcpyHostToDevice, st));
        PAT_CUDA(cudaMemcpyAsync(F(b, TKM), g[b]->pc.tile_kmax, sz[TKM], cudaMemcpyDeviceToDevice, st));
        PAT_CUDA(cudaMemsetAsync(buf(b, KT), 0, NN * 8, st));
    }
    int* stopped = nullptr;
    void* dev = nullptr;
    if (!rc) rc = cudaMallocAsync((void**)&stopped, sizeof(int), st) == cudaSuccess &&
                          cudaMemsetAsync(stopped, 0, sizeof(int), st) == cudaSuccess
                      ? PAT_OK
                      : fail(PAT_ERR_CUDA, std::string(who) + ": stop counter");
    // device argument blocks: K and K^T per problem, as the batch engine's
    std::vector<char> host;
    Arena ar(host);
    size_t fw_off[2] = {0, 0}, ad_off[2] = {0, 0}, fg_off = 0, fi_off = 0, amap_off = 0, finmap_off = 0;
    GapPlan gp;
    int n_adj = 0;
    if (!rc) {
        std::vector<FwdArgs> fw[2], fg;
        std::vector<AdjArgs> ad[2];
        std::vector<FinalArgs> fi;
        std::vector<std::pair<float, int2>> order;
        std::vector<Prob> prs(B);
        for (int b = 0; b < B; ++b) {
            InfoDev* in = inf(b);
            for (int par = 0; par < 2; ++par) {
                FwdArgs fa = make_fwd_args(g[b], F(b, UBAR));
                fa.q = F(b, Q);
                fa.f = f[b];
                fa.sig_q = F(b, SIGQ);
                fa.sig_scalar = -1.f;
                fa.step_mul = in->step_mul;
                fa.qw = F(b, QW);
                fa.qmax_bits = &in->qmax_bits[par];
                fa.stop = &in->stop;
                fw[par].push_back(fa);
                ad[par].push_back(make_adj_args(g[b], F(b, Q), F(b, QW), &in->qmax_bits[par],
                                                (int*)buf(b, KT) + (size_t)par * NN, &in->stop));
            }
            FwdArgs ga = make_fwd_args(g[b], F(b, U));
            ga.q = F(b, Q);
            ga.f = f[b];
            ga.partials = (double*)buf(b, DPART);
            ga.stop = &in->stop;
            fg.push_back(ga);
            fi.push_back(FinalArgs{(double*)buf(b, DPART), g[b]->fwd_n_ctas, (double*)buf(b, PPART), n_pix, p[b].alpha,
                                   0.0, p[b].box_u, p[b].box_v, p[b].tol, PAT_WAV, PAT_ADAPT_NONE, in, stopped});
            for (int i = 0; i < g[b]->adj_items; ++i) order.push_back({g[b]->adj_item_cost[i], make_int2(b, i)});
            prs[b].g = g[b];
        }
        for (int par = 0; par < 2; ++par) {
            fw_off[par] = ar.put(fw[par].data(), fw[par].size());
            ad_off[par] = ar.put(ad[par].data(), ad[par].size());
        }
        fg_off = ar.put(fg.data(), fg.size());
        fi_off = ar.put(fi.data(), fi.size());
        forward_groups(prs.data(), B, ar, gp);
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<float, int2>& x, const std::pair<float, int2>& y) { return x.first > y.first; });
        std::vector<int2> am, fin;
        for (auto& e : order) am.push_back(e.second);
        n_adj = (int)am.size();
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < GAP_FINAL_BLOCKS; ++i) fin.push_back(make_int2(b, i));
        amap_off = ar.put(am.data(), am.size());
        finmap_off = ar.put(fin.data(), fin.size());
        rc = ar.upload(&dev, st);
    }
    const char* base = (const char*)dev;
    // the wavelet kernels take problem 0's pointers; problem b's lie b * ps bytes on
    float *u = F(0, U), *u_old = F(0, UOLD), *ubar = F(0, UBAR), *r = F(0, R), *wb = F(0, WB), *wtr = F(0, WTR);
    float *scr = F(0, SCR), *scr2 = F(0, SCR2), *wu = F(0, WU), *tau = F(0, TAU), *sigr = F(0, SIGR);
    float *scrt = F(0, SCRT), *scal = F(0, SCAL);
    int* kt = (int*)buf(0, KT);
    double* ppart = (double*)buf(0, PPART);
    InfoDev* in = inf(0);
    const int tiles_x = g[0]->adj_tiles_x;
    auto iteration = [&](int it, bool gap, cudaStream_t s) -> int {
        const int par = it & 1;
        int e = launch_forward_groups(FWD_PROX, (const FwdArgs*)(base + fw_off[par]), gp, base, s);
        if (cwt) {
            if (!e) e = launch_cwt_analysis(ubar, N, J, wm.bank, wb, scr, &in->stop, s, B, ps);
            if (!e) e = launch_cwt_dual(r, wb, sigr, in->step_mul, scal, N, J, &in->stop, s, B, ps);
        } else {
            if (!e) e = launch_wav_analysis(ubar, N, J, wb, scr, &in->stop, s, B, ps);
            if (!e) e = launch_wav_dual(r, wb, sigr, in->step_mul, scal, NN, &in->stop, s, B, ps);
        }
        if (!e)
            e = launch_adjoint_b((const AdjArgs*)(base + ad_off[par]), (const int2*)(base + amap_off), n_adj, true, s);
        if (cwt) {
            if (!e) e = launch_cwt_uncombine(r, scrt, N, J, &in->stop, s, B, ps);
            if (!e) e = launch_cwt_synthesis(scrt, N, J, wm.bank, wtr, scr, &in->stop, s, B, ps);
        } else {
            if (!e) e = launch_wav_synthesis(r, N, J, wtr, scr, &in->stop, s, B, ps);
        }
        WavPrimalArgs pa;
        pa.n = N;
        pa.scal = scal;
        pa.tau_u = tau;
        pa.step_mul = in->step_mul;
        pa.kt = KtView{kt + (size_t)par * NN, &in->qmax_bits[par], F(0, TKM), tiles_x};
        pa.wtr = wtr;
        pa.u = u;
        pa.u_old = gap ? u_old : nullptr;
        pa.ubar = ubar;
        pa.kt_clear = kt + (size_t)(1 - par) * NN;
        pa.qmax_next = &in->qmax_bits[1 - par];
        pa.stop = &in->stop;
        pa.iter = &in->iter;
        if (!e) e = launch_wav_primal(pa, s, B, ps);
        if (gap && !e) {
            e = cwt ? launch_cwt_analysis(u, N, J, wm.bank, wu, scr2, &in->stop, s, B, ps)
                    : launch_wav_analysis(u, N, J, wu, scr2, &in->stop, s, B, ps);
            if (!e) e = launch_forward_groups(FWD_GAP, (const FwdArgs*)(base + fg_off), gp, base, s);
            if (cwt) {
                CwtGapArgs cg{N, GAP_PIX_TERMS, N >> J, wu, pa.kt, wtr, u, u_old, ppart, &in->stop};
                if (!e) e = launch_cwt_gap_pixels(cg, n_pix, s, B, ps);
            } else {
                WavGapArgs wg{N, GAP_PIX_TERMS, wu, pa.kt, wtr, u, u_old, ppart, &in->stop};
                if (!e) e = launch_wav_gap_pixels(wg, n_pix, s, B, ps);
            }
            if (!e) {
                k_gap_final_b<<<B * GAP_FINAL_BLOCKS, GAP_FINAL_THREADS, 0, s>>>((const FinalArgs*)(base + fi_off),
                                                                                (const int2*)(base + finmap_off));
                count_launch();
                if (cudaGetLastError() != cudaSuccess) e = fail(PAT_ERR_CUDA, "k_gap_final_b");
            }
        }
        return e;
    };
    const int iters = p[0].iters, ge = p[0].gap_every;
    bool can_stop = false;
    for (int k = 0; k < B; ++k) can_stop = can_stop || p[k].tol > 0;
    if (!rc && iters > 0) {
        auto gap_due = [&](int it) { return (ge > 0 && (it + 1) % ge == 0) || it + 1 == iters; };
        const int P = ge > 0 ? (ge % 2 == 0 ? ge : 2 * ge) : 2;
        const int nper = (iters - 1) / P;
        int start = 0;
        bool all_stopped = false;
        if (!prof_on() && nper >= 2) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaStream_t ls = loop_stream();
            cudaEvent_t fork = nullptr, join = nullptr;
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
            cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
            cudaEventRecord(fork, st);
            cudaStreamWaitEvent(ls, fork, 0);
            const long long l0 = pat_kernel_launches();
            cudaError_t ce = cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal);
            for (int it = 0; it < P && !rc && ce == cudaSuccess; ++it) rc = iteration(it, ge > 0 && (it + 1) % ge == 0, ls);
            cudaError_t e2 = cudaStreamEndCapture(ls, &graph);
            if (ce == cudaSuccess) ce = e2;
            if (!rc && ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
            const long long per_period = pat_kernel_launches() - l0;
            int* snap = can_stop ? stop_snapshots() : nullptr;
            cudaEvent_t ev[2] = {nullptr, nullptr};
            bool pending[2] = {false, false};
            if (snap)
                for (int i = 0; i < 2 && ce == cudaSuccess; ++i) ce = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
            int launched = 0;
            constexpr int CHUNK = 8;
            for (int chunk = 0; !rc && ce == cudaSuccess && launched < nper; ++chunk) {
                const int n = std::min(CHUNK, nper - launched);
                for (int k = 0; k < n && ce == cudaSuccess; ++k) ce = cudaGraphLaunch(exec, ls);
                launched += n;
                if (!snap || ce != cudaSuccess) continue;
                const int cur = chunk & 1, prev = cur ^ 1;
                ce = cudaMemcpyAsync(&snap[cur], stopped, sizeof(int), cudaMemcpyDeviceToHost, ls);
                if (ce == cudaSuccess) ce = cudaEventRecord(ev[cur], ls);
                pending[cur] = ce == cudaSuccess;
                if (pending[prev] && ce == cudaSuccess) {
                    ce = cudaEventSynchronize(ev[prev]);
                    pending[prev] = false;
                    if (ce == cudaSuccess && *(volatile int*)&snap[prev] >= B) {
                        all_stopped = true;
                        break;
                    }
                }
            }
            for (int i = 0; i < 2; ++i)
                if (ev[i]) {
                    if (pending[i]) cudaEventSynchronize(ev[i]);
                    cudaEventDestroy(ev[i]);
                }
            for (int k = 1; k < launched; ++k)
                for (long long c = 0; c < per_period; ++c) count_launch();
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            cudaEventRecord(join, ls);
            cudaStreamWaitEvent(st, join, 0);
            cudaEventDestroy(fork);
            cudaEventDestroy(join);
            if (!rc && ce != cudaSuccess) rc = cuda_fail(ce, "run_wavelet: graph");
            start = nper * P;
        }
        for (int it = start; !rc && !all_stopped && it < iters; ++it) rc = iteration(it, gap_due(it), st);
    }
    // outputs: u, x = [u], xbar = [ubar], y = [q, r]
    for (int b = 0; b < B && !rc; ++b) {
        const pat_params& pb = p[b];
        const long long Sb = (long long)g[b]->desc.n_det * g[b]->desc.n_t;
        PAT_CUDA(cudaMemcpyAsync(u_out[b], F(b, U), NN * 4, cudaMemcpyDeviceToDevice, st));
        if (pb.x_out_dev) PAT_CUDA(cudaMemcpyAsync(pb.x_out_dev, F(b, U), NN * 4, cudaMemcpyDeviceToDevice, st));
        if (pb.x_lo_out_dev) PAT_CUDA(cudaMemsetAsync(pb.x_lo_out_dev, 0, NN * 4, st));
        if (pb.xbar_out_dev) PAT_CUDA(cudaMemcpyAsync(pb.xbar_out_dev, F(b, UBAR), NN * 4, cudaMemcpyDeviceToDevice, st));
        if (pb.y_out_dev) {
            PAT_CUDA(cudaMemcpyAsync(pb.y_out_dev, F(b, Q), Sb * 4, cudaMemcpyDeviceToDevice, st));
            PAT_CUDA(cudaMemcpyAsync(pb.y_out_dev + Sb, F(b, R), NR * 4, cudaMemcpyDeviceToDevice, st));
        }
    }
    std::vector<InfoDev> h(B);
    for (int b = 0; b < B && !rc; ++b)
        rc = cudaMemcpyAsync(&h[b], inf(b), sizeof(InfoDev), cudaMemcpyDeviceToHost, st) == cudaSuccess ? 0 : PAT_ERR_CUDA;
    cudaEventRecord(e1, st);
    if (dev) cudaFreeAsync(dev, st);
    if (stopped) cudaFreeAsync(stopped, st);
    cudaFreeAsync(ws, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (!rc && se != cudaSuccess) rc = cuda_fail(se, who);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    prof_collect();
    if (rc) return rc;
    bool diverged = false;
    for (int b = 0; b < B; ++b) {
        if (infos) {
            pat_info& io = infos[b];
            io.iters_done = iters == 0 ? 0 : h[b].iters_done;
            io.status = h[b].stop ? h[b].status : PAT_STATUS_MAXITER;
            io.primal = h[b].primal;
            io.dual = h[b].dual;
            io.gap = h[b].gap;
            io.rel_gap = h[b].rel_gap;
            io.residual = h[b].residual;
            io.ms = ms;
            io.step_ratio = (double)h[b].step_mul[0];
        }
        diverged = diverged || h[b].status == PAT_STATUS_DIVERGED;
    }
    if (diverged) return fail(PAT_ERR_NONFINITE, std::string(who) + ": duality gap not finite");
    return PAT_OK;
}

static int run_batch(int B, const pat_geometry* const* g, const float* const* f, const pat_params* p,
                     float* const* u_out, pat_info* infos, cudaStream_t st, const char* who) {
    if (B == 0) return PAT_OK;
    for (int b = 0; b < B; ++b)
        if (p[b].reg == PAT_WAV) return fail(PAT_ERR_INVALID_ARG, std::string(who) + ": PAT_WAV has no batch engine");
    for (int b = 1; b < B; ++b)
        if (p[b].iters != p[0].iters || p[b].gap_every != p[0].gap_every)
            return fail(PAT_ERR_INVALID_ARG, std::string(who) + ": a batch needs equal iters and gap_every");
    cudaEvent_t e0, e1, fork, join;
    PAT_CUDA(cudaEventCreate(&e0));
    PAT_CUDA(cudaEventCreate(&e1));
    PAT_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    PAT_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    PAT_CUDA(cudaEventRecord(e0, st));
    std::vector<Prob> pr(B);
    int rc = PAT_OK;
    for (int b = 0; b < B && !rc; ++b) {
        pr[b].g = g[b];
        pr[b].f = f[b];
        pr[b].p = p[b];
        pr[b].u_out = u_out[b];
        rc = init_problem(pr[b], st);
    }
    std::vector<char> host;
    void* dev = nullptr;
    int* stopped = nullptr;
    bool can_stop = false;
    for (int b = 0; b < B; ++b) can_stop = can_stop || p[b].tol > 0;
    if (!rc && p[0].iters > 0) {
        rc = cudaMallocAsync((void**)&stopped, sizeof(int), st) == cudaSuccess &&
                     cudaMemsetAsync(stopped, 0, sizeof(int), st) == cudaSuccess
                 ? PAT_OK
                 : fail(PAT_ERR_CUDA, std::string(who) + ": stop counter");
    }
    if (!rc && p[0].iters > 0) {
        Arena ar(host);
        IterPlan ip;
        build_iter_plan(pr.data(), B, ar, ip, stopped);
        rc = ar.upload(&dev, st);
        cudaStream_t ls = loop_stream();
        if (!ls) rc = fail(PAT_ERR_CUDA, std::string(who) + ": no loop stream");
        if (!rc) rc = cudaEventRecord(fork, st) == cudaSuccess ? PAT_OK : PAT_ERR_CUDA;
        if (!rc) rc = cudaStreamWaitEvent(ls, fork, 0) == cudaSuccess ? PAT_OK : PAT_ERR_CUDA;
        if (!rc) rc = run_iterations(ip, (const char*)dev, p[0].iters, p[0].gap_every, ls, stopped, B, can_stop);
        if (ls) {
            cudaEventRecord(join, ls);
            cudaStreamWaitEvent(st, join, 0);
        }
    }
    for (int b = 0; b < B && !rc; ++b) rc = finish_problem(pr[b], st);
    std::vector<InfoDev> hinfo(B);
    for (int b = 0; b < B && !rc; ++b)
        rc = cudaMemcpyAsync(&hinfo[b], pr[b].ws.info, sizeof(InfoDev), cudaMemcpyDeviceToHost, st) ? PAT_ERR_CUDA : 0;
    cudaEventRecord(e1, st);
    if (dev) cudaFreeAsync(dev, st);
    if (stopped) cudaFreeAsync(stopped, st);
    for (int b = 0; b < B; ++b)
        if (pr[b].ws.base) cudaFreeAsync(pr[b].ws.base, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (!rc && se != cudaSuccess) rc = cuda_fail(se, std::string(who).c_str());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    prof_collect();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    if (rc) {
        if (rc == PAT_ERR_CUDA && std::string(pat_last_error()).empty())
            set_error(std::string(who) + ": " + cudaGetErrorString(cudaGetLastError()));
        return rc;
    }
    bool diverged = false;
    for (int b = 0; b < B; ++b) {
        const InfoDev& h = hinfo[b];
        if (infos) {
            pat_info& in = infos[b];
            in.iters_done = p[b].iters == 0 ? 0 : h.iters_done;
            in.status = h.stop ? h.status : PAT_STATUS_MAXITER;
            in.primal = h.primal;
            in.dual = h.dual;
            in.gap = h.gap;
            in.rel_gap = h.rel_gap;
            in.residual = h.residual;
            in.ms = ms;
            in.step_ratio = (double)h.step_mul[0];
        }
        diverged = diverged || h.status == PAT_STATUS_DIVERGED;
    }
    if (diverged) return fail(PAT_ERR_NONFINITE, std::string(who) + ": duality gap not finite");
    return PAT_OK;
}

// ---------------------------------------------------------------------------------
// Phase timing: the batch runs its iterations as usual, then each phase's launch (all
// problems, iteration parity 0) is captured `reps` times in a graph of its own and
// replayed between two CUDA events.  Launches of one graph follow each other with no
// host work in between, as in the iteration loop's graph, so the per-launch times add up
// to the loop's time per iteration.  Repeated K^T launches accumulate without the clear
// that an iteration performs (integer wrap-around, same work), so the state is not used
// afterwards and nothing is written to the caller's buffers.
// ---------------------------------------------------------------------------------
static int time_phases(int B, const pat_geometry* const* g, const float* const* f, const pat_params* p, int reps,
                       double* us, cudaStream_t st, const char* who) {
    std::vector<Prob> pr(B);
    int rc = PAT_OK;
    for (int b = 0; b < B && !rc; ++b) {
        pr[b].g = g[b];
        pr[b].f = f[b];
        pr[b].p = p[b];
        pr[b].p.tol = 0.0;
        pr[b].p.adapt = PAT_ADAPT_NONE;
        pr[b].p.x_out_dev = pr[b].p.xbar_out_dev = pr[b].p.y_out_dev = pr[b].p.x_lo_out_dev = nullptr;
        rc = init_problem(pr[b], st);
    }
    std::vector<char> host;
    void* dev = nullptr;
    cudaStream_t ls = loop_stream();
    cudaEvent_t fork = nullptr, join = nullptr, e0 = nullptr, e1 = nullptr;
    if (!rc && !ls) rc = fail(PAT_ERR_CUDA, std::string(who) + ": no loop stream");
    if (!rc) rc = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
                          cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess &&
                          cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess
                      ? PAT_OK
                      : fail(PAT_ERR_CUDA, std::string(who) + ": events");
    IterPlan ip;
    if (!rc) {
        Arena ar(host);
        build_iter_plan(pr.data(), B, ar, ip, nullptr);
        rc = ar.upload(&dev, st);
    }
    if (!rc) rc = cudaEventRecord(fork, st) == cudaSuccess && cudaStreamWaitEvent(ls, fork, 0) == cudaSuccess
                      ? PAT_OK
                      : fail(PAT_ERR_CUDA, std::string(who) + ": stream join");
    const char* base = (const char*)dev;
    if (!rc) rc = run_iterations(ip, base, p[0].iters, p[0].gap_every, ls, nullptr, B, false);
    for (int ph = 0; ph < PAT_NPHASES; ++ph) us[ph] = 0.0;
    // state-preserving phases first; K^T (accumulates) and the update (reads it) last
    const int order[4] = {PAT_PHASE_FORWARD_PROX, PAT_PHASE_GAP, PAT_PHASE_ADJOINT, PAT_PHASE_UPDATE};
    for (int oi = 0; oi < 4 && !rc; ++oi) {
        const int ph = order[oi];
        auto enqueue = [&]() -> int {
            if (ph == PAT_PHASE_FORWARD_PROX)
                return launch_forward_groups(FWD_PROX, (const FwdArgs*)(base + ip.fwd[0]), ip.gp, base, ls);
            if (ph == PAT_PHASE_ADJOINT)
                return launch_adjoint_b((const AdjArgs*)(base + ip.adj[0]), (const int2*)(base + ip.map_adj), ip.n_adj,
                                        true, ls);
            if (ph == PAT_PHASE_UPDATE) {
                const UpdateArgs* ua = (const UpdateArgs*)(base + ip.upd[0][0]);
                for (int r = 0; r < 3; ++r)
                    for (int t = 0; t < UPD_TILES; ++t) {
                        const int e = launch_update_b(r, t, ua, (const int2*)(base + ip.map_upd[r][t]), ip.n_upd[r][t], ls);
                        if (e) return e;
                    }
                return PAT_OK;
            }
            return launch_gap_phase((const FwdArgs*)(base + ip.fgap[0]), (const GapArgs*)(base + ip.gpix[0]),
                                    (const FinalArgs*)(base + ip.fin), ip.gp, base, ls);
        };
        for (int b = 0; b < B; ++b) cudaMemsetAsync(&pr[b].ws.info->stop, 0, sizeof(int), ls);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const long long l0 = pat_kernel_launches();
        cudaError_t e = cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "time_phases: capture");
            break;
        }
        for (int r = 0; r < reps && !rc; ++r) rc = enqueue();
        e = cudaStreamEndCapture(ls, &graph);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "time_phases: capture");
        if (!rc) {
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) rc = cuda_fail(e, "time_phases: instantiate");
        }
        const long long per_graph = pat_kernel_launches() - l0;
        if (!rc) {
            e = cudaGraphLaunch(exec, ls);   // warm-up replay
            if (e == cudaSuccess) e = cudaEventRecord(e0, ls);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, ls);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ls);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) rc = cuda_fail(e, "time_phases: replay");
            us[ph] = 1e3 * (double)ms / reps;
            for (long long k = 0; k < per_graph; ++k) count_launch();   // the second replay
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    if (join && ls) {
        cudaEventRecord(join, ls);
        cudaStreamWaitEvent(st, join, 0);
    }
    if (dev) cudaFreeAsync(dev, st);
    for (int b = 0; b < B; ++b)
        if (pr[b].ws.base) cudaFreeAsync(pr[b].ws.base, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (!rc && se != cudaSuccess) rc = cuda_fail(se, who);
    for (cudaEvent_t ev : {fork, join, e0, e1})
        if (ev) cudaEventDestroy(ev);
    return rc;
}

// ---------------------------------------------------------------------------------
// Launch-shape autotuner: per geometry, each kernel's candidate shapes are timed on the
// problem itself (phase timing in graphs, as pat_time_phases), one kernel at a time with
// the others at their current choice, and the fastest is kept.  Choices are cached in a
// JSON file keyed by (N, D, T, M, regulariser, GPU name).
// ---------------------------------------------------------------------------------
struct ShapeEntry {
    std::string key;
    pat_shapes s;
    double us[3];   // K, K^T, update: microseconds per launch of the chosen shapes
};

static std::string shape_key(const pat_geometry* g, int reg) {
    cudaDeviceProp prop;
    std::string gpu = "unknown";
    if (cudaGetDeviceProperties(&prop, g->device) == cudaSuccess) gpu = prop.name;
    else cudaGetLastError();
    for (char& c : gpu)
        if (c == '"' || c == '\\') c = '_';
    char buf[160];
    snprintf(buf, sizeof buf, "N=%d D=%d T=%d M=%d reg=%d", g->desc.n, g->desc.n_det, g->desc.n_t, g->desc.quad_m, reg);
    return std::string(buf) + " gpu=" + gpu;
}

// The cache holds one entry per line inside {"entries": [ ... ]}; lines that do not parse
// are ignored.
static std::vector<ShapeEntry> read_shape_cache(const char* path) {
    std::vector<ShapeEntry> out;
    FILE* fp = path ? fopen(path, "r") : nullptr;
    if (!fp) return out;
    char line[1024];
    while (fgets(line, sizeof line, fp)) {
        const char* k = strstr(line, "\"key\": \"");
        if (!k) continue;
        k += 8;
        const char* e = strchr(k, '"');
        if (!e) continue;
        ShapeEntry se;
        se.key.assign(k, e);
        if (sscanf(e, "\", \"forward\": %d, \"adjoint_waves\": %d, \"update_tile\": %d, \"us\": [%lf, %lf, %lf]",
                   &se.s.forward, &se.s.adjoint_waves, &se.s.update_tile, &se.us[0], &se.us[1], &se.us[2]) == 6)
            out.push_back(se);
    }
    fclose(fp);
    return out;
}

static int write_shape_cache(const char* path, const std::vector<ShapeEntry>& entries) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE* fp = fopen(tmp.c_str(), "w");
    if (!fp) return fail(PAT_ERR_INVALID_ARG, std::string("pat_tune_shapes: cannot write ") + tmp);
    fprintf(fp, "{\"entries\": [\n");
    for (size_t i = 0; i < entries.size(); ++i) {
        const ShapeEntry& se = entries[i];
        fprintf(fp, "  {\"key\": \"%s\", \"forward\": %d, \"adjoint_waves\": %d, \"update_tile\": %d, \"us\": [%.3f, %.3f, %.3f]}%s\n",
                se.key.c_str(), se.s.forward, se.s.adjoint_waves, se.s.update_tile, se.us[0], se.us[1], se.us[2],
                i + 1 < entries.size() ? "," : "");
    }
    fprintf(fp, "]}\n");
    const bool ok = fclose(fp) == 0;
    if (!ok || rename(tmp.c_str(), path) != 0) return fail(PAT_ERR_INVALID_ARG, std::string("pat_tune_shapes: cannot write ") + path);
    return PAT_OK;
}

static int tune_one(pat_geometry* g, const float* f, const pat_params* p, int reps, cudaStream_t st, ShapeEntry& se) {
    pat_params q = *p;
    q.iters = 20;
    q.gap_every = 10;
    q.tol = 0.0;
    q.adapt = PAT_ADAPT_NONE;
    q.x_out_dev = q.xbar_out_dev = q.y_out_dev = q.x_lo_out_dev = nullptr;
    const pat_geometry* gc = g;
    double us[PAT_NPHASES];
    pat_shapes cur = g->shapes;
    auto time_with = [&](const pat_shapes& s) -> int {
        int rc = pat_geometry_set_shapes(g, &s);
        if (!rc) rc = time_phases(1, &gc, &f, &q, reps, us, st, "pat_tune_shapes");
        return rc;
    };
    // K: the slab variants and the global one (variants that resolve alike are timed once)
    double best = 1e300;
    pat_shapes best_s = cur;
    std::vector<int> seen;
    for (int fv : {PAT_FWD_SLAB_TWO, PAT_FWD_SLAB_ONE, PAT_FWD_GLOBAL}) {
        pat_shapes s = best_s;
        s.forward = fv;
        int rc = pat_geometry_set_shapes(g, &s);
        if (rc) return rc;
        const int resolved = g->shapes.forward;
        if (std::find(seen.begin(), seen.end(), resolved) != seen.end()) continue;
        seen.push_back(resolved);
        rc = time_phases(1, &gc, &f, &q, reps, us, st, "pat_tune_shapes");
        if (rc) return rc;
        if (us[PAT_PHASE_FORWARD_PROX] < best) {
            best = us[PAT_PHASE_FORWARD_PROX];
            best_s = g->shapes;
        }
    }
    se.us[0] = best;
    // K^T: work items filling one or two waves
    best = 1e300;
    pat_shapes k_best = best_s;
    for (int w : {1, 2}) {
        pat_shapes s = k_best;
        s.adjoint_waves = w;
        const int rc = time_with(s);
        if (rc) return rc;
        if (us[PAT_PHASE_ADJOINT] < best) {
            best = us[PAT_PHASE_ADJOINT];
            best_s = g->shapes;
        }
    }
    se.us[1] = best;
    // fused update tile
    best = 1e300;
    k_best = best_s;
    for (int t = 0; t < UPD_TILES; ++t) {
        pat_shapes s = k_best;
        s.update_tile = t;
        const int rc = time_with(s);
        if (rc) return rc;
        if (us[PAT_PHASE_UPDATE] < best) {
            best = us[PAT_PHASE_UPDATE];
            best_s = g->shapes;
        }
    }
    se.us[2] = best;
    se.s = best_s;
    return pat_geometry_set_shapes(g, &best_s);
}

// ---------------------------------------------------------------------------------
// paper rule (Sec. 3.3.2): L1 = ||K||, L2 = ||B|| by power iteration from the start
// vector x_j = 1 + sin(0.7 j + 0.3)/2; tau = 1/L1, sigma_i = 0.99 / (4 tau L_i^2)
// ---------------------------------------------------------------------------------
__global__ void k_power_start(float* x, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) x[i] = (float)(1.0 + 0.5 * sin(0.7 * (double)i + 0.3));
}

__global__ void k_norm2(const float* __restrict__ x, long long n, double* out) {
    double v[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[0] += (double)x[i] * x[i];
    block_sum<1>(v);
    if (threadIdx.x == 0) atomicAdd(out, v[0]);
}

__global__ void k_scale(float* x, long long n, const double* nrm2, double* lam_out) {
    const double nr = sqrt(*nrm2);
    if (blockIdx.x == 0 && threadIdx.x == 0 && lam_out) *lam_out = nr;
    const float s = nr > 0 ? (float)(1.0 / nr) : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= s;
}

// B x for the regulariser block of A: x = (u[, v1, v2]), out rows as in pat_params y.
__global__ void k_apply_B(int N, int reg, float gamma, const float* __restrict__ xi, const float* __restrict__ x,
                          float* __restrict__ out) {
    const long long NN = (long long)N * N;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= N || gy >= N) return;
    const int gi = gy * N + gx;
    const bool ax = gx < N - 1, by = gy < N - 1, axm = gx >= 1, bym = gy >= 1;
    float g0 = ax ? x[gi + 1] - x[gi] : 0.f, g1 = by ? x[gi + N] - x[gi] : 0.f;
    if (reg == PAT_DTV) {
        float o0, o1;
        dxi_apply(xi[gi], xi[NN + gi], gamma, g0, g1, o0, o1);
        g0 = o0;
        g1 = o1;
    }
    if (reg == PAT_TGV) {
        g0 -= x[NN + gi];
        g1 -= x[2 * NN + gi];
        auto v = [&](int c, int xx, int yy) { return x[(1 + c) * NN + yy * N + xx]; };
        const float v1 = ax ? v(0, gx, gy) : 0.f, v1l = axm ? v(0, gx - 1, gy) : 0.f;
        const float v2 = by ? v(1, gx, gy) : 0.f, v2d = bym ? v(1, gx, gy - 1) : 0.f;
        const float v1y = by ? v(0, gx, gy) : 0.f, v1d = bym ? v(0, gx, gy - 1) : 0.f;
        const float v2x = ax ? v(1, gx, gy) : 0.f, v2l = axm ? v(1, gx - 1, gy) : 0.f;
        out[2 * NN + gi] = v1 - v1l;
        out[3 * NN + gi] = v2 - v2d;
        out[4 * NN + gi] = ((v1y - v1d) + (v2x - v2l)) * kInvSqrt2f;
    }
    out[gi] = g0;
    out[NN + gi] = g1;
}

// B^T y
__global__ void k_apply_BT(int N, int reg, float gamma, const float* __restrict__ xi, const float* __restrict__ y,
                           float* __restrict__ out) {
    const long long NN = (long long)N * N;
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= N || gy >= N) return;
    const int gi = gy * N + gx;
    const bool ax = gx < N - 1, by = gy < N - 1;
    auto rm = [&](int c, int xx, int yy) -> float {
        if (xx < 0 || yy < 0) return 0.f;
        if (c == 0 && xx >= N - 1) return 0.f;
        if (c == 1 && yy >= N - 1) return 0.f;
        float r0 = y[yy * N + xx], r1 = y[NN + yy * N + xx];
        if (reg == PAT_DTV) {
            float o0, o1;
            dxi_apply(xi[yy * N + xx], xi[NN + yy * N + xx], gamma, r0, r1, o0, o1);
            r0 = o0;
            r1 = o1;
        }
        return c == 0 ? r0 : r1;
    };
    const float divr = rm(0, gx, gy) - rm(0, gx - 1, gy) + rm(1, gx, gy) - rm(1, gx, gy - 1);
    out[gi] = -divr;
    if (reg == PAT_TGV) {
        auto s = [&](int c, int xx, int yy) { return y[(2 + c) * NN + yy * N + xx]; };
        const float dx11 = ax ? s(0, gx + 1, gy) - s(0, gx, gy) : 0.f;
        const float dy12 = by ? s(2, gx, gy + 1) - s(2, gx, gy) : 0.f;
        const float dy22 = by ? s(1, gx, gy + 1) - s(1, gx, gy) : 0.f;
        const float dx12 = ax ? s(2, gx + 1, gy) - s(2, gx, gy) : 0.f;
        out[NN + gi] = -dx11 - dy12 * kInvSqrt2f - y[gi];
        out[2 * NN + gi] = -dy22 - dx12 * kInvSqrt2f - y[NN + gi];
    }
}

static constexpr int kPowerIters = 100;

int scalar2_steps(const pat_geometry* g, const pat_params* p, ScalarSteps& out, cudaStream_t st) {
    const int N = g->desc.n;
    const long long NN = (long long)N * N, S = (long long)g->desc.n_det * g->desc.n_t;
    const long long nx = NN * (p->reg == PAT_TGV ? 3 : 1), ny = NN * (p->reg == PAT_TGV ? 5 : 2);
    float *x = nullptr, *y = nullptr;
    double* acc = nullptr;
    PAT_CUDA(cudaMallocAsync(&x, (size_t)std::max(nx, NN) * 4, st));
    PAT_CUDA(cudaMallocAsync(&y, (size_t)std::max(ny, S) * 4, st));
    PAT_CUDA(cudaMallocAsync(&acc, 2 * kPowerIters * 2 * sizeof(double), st));
    PAT_CUDA(cudaMemsetAsync(acc, 0, 2 * kPowerIters * 2 * sizeof(double), st));
    dim3 blk(32, 8), grd(ceil_div(N, 32), ceil_div(N, 8));
    const int nb = 2 * sm_count();
    double lam[2] = {0, 0};
    for (int op = 0; op < 2; ++op) {
        const long long n = op == 0 ? NN : nx;
        k_power_start<<<ceil_div(n, 256), 256, 0, st>>>(x, n); count_launch();
        double* a0 = acc + op * 2 * kPowerIters;
        k_norm2<<<nb, 256, 0, st>>>(x, n, a0); count_launch();
        k_scale<<<nb, 256, 0, st>>>(x, n, a0, nullptr); count_launch();
        for (int it = 0; it < kPowerIters; ++it) {
            if (op == 0) {
                int rc = launch_forward(g, x, y, st);
                if (rc) return rc;
                rc = launch_adjoint(g, y, x, st);
                if (rc) return rc;
            } else {
                k_apply_B<<<grd, blk, 0, st>>>(N, p->reg, (float)p->gamma, p->xi_dev, x, y); count_launch();
                k_apply_BT<<<grd, blk, 0, st>>>(N, p->reg, (float)p->gamma, p->xi_dev, y, x); count_launch();
            }
            double* slot = a0 + 1 + it;
            k_norm2<<<nb, 256, 0, st>>>(x, n, slot); count_launch();
            k_scale<<<nb, 256, 0, st>>>(x, n, slot, nullptr); count_launch();
        }
        PAT_LAUNCH_CHECK("power iteration");
        double last = 0;
        PAT_CUDA(cudaMemcpyAsync(&last, a0 + kPowerIters, sizeof(double), cudaMemcpyDeviceToHost, st));
        PAT_CUDA(cudaStreamSynchronize(st));
        lam[op] = sqrt(sqrt(last));  // ||A^T A x|| -> sigma^2
    }
    cudaFreeAsync(x, st);
    cudaFreeAsync(y, st);
    cudaFreeAsync(acc, st);
    const double L1 = lam[0], L2 = lam[1];
    if (!(L1 > 0) || !(L2 > 0)) return fail(PAT_ERR_INVALID_ARG, "pat_reconstruct: zero operator norm");
    const double tau = 1.0 / L1;
    out.tau = (float)tau;
    out.sig_q = (float)(0.99 / (4.0 * tau * L1 * L1));
    out.sig2 = (float)(0.99 / (4.0 * tau * L2 * L2));
    return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" void pat_params_default(pat_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->reg = PAT_TV;
    p->alpha = 0.05;
    p->beta = 1.0;
    p->gamma = 0.95;
    p->iters = 100;
    p->tol = 0.0;
    p->gap_every = 10;
    p->precond = PAT_PRECOND_DIAG;
    p->theta = 1.0;
    p->box_u = 2.0;
    p->box_v = 4.0;
    p->step_ratio = 1.0;
    p->adapt = PAT_ADAPT_NONE;
    p->wavelet_levels = 4;
}

extern "C" int pat_reconstruct(const pat_geometry* g, const float* f_dev, const pat_params* p, float* u_dev,
                               pat_info* info, void* stream) {
    int rc = validate(g, p, "pat_reconstruct");
    if (rc) return rc;
    if (!f_dev || !u_dev) return fail(PAT_ERR_INVALID_ARG, "pat_reconstruct: NULL data or output");
    if (p->reg == PAT_WAV) return run_wavelet(1, &g, &f_dev, p, &u_dev, info, (cudaStream_t)stream, "pat_reconstruct");
    return run_batch(1, &g, &f_dev, p, &u_dev, info, (cudaStream_t)stream, "pat_reconstruct");
}

extern "C" int pat_reconstruct_batched(int count, const pat_geometry* const* g, const float* const* f_dev,
                                       const pat_params* p, float* const* u_dev, pat_info* infos, void* stream) {
    if (count < 0 || (count > 0 && (!g || !f_dev || !p || !u_dev)))
        return fail(PAT_ERR_INVALID_ARG, "pat_reconstruct_batched: NULL arrays");
    for (int i = 0; i < count; ++i) {
        int rc = validate(g[i], &p[i], "pat_reconstruct_batched");
        if (rc) return rc;
        if (!f_dev[i] || !u_dev[i]) return fail(PAT_ERR_INVALID_ARG, "pat_reconstruct_batched: NULL data or output");
    }
    // problems advance in lockstep: those sharing (iters, gap_every) run as one batch, the
    // wavelet problems among them in batches that also share N and the transform
    std::vector<char> done(count, 0);
    for (int i = 0; i < count; ++i) {
        if (done[i]) continue;
        std::vector<int> idx;
        for (int j = i; j < count; ++j)
            if (!done[j] && p[j].iters == p[i].iters && p[j].gap_every == p[i].gap_every &&
                (p[i].reg == PAT_WAV) == (p[j].reg == PAT_WAV) &&
                (p[i].reg != PAT_WAV || wav_same_batch(g[i], &p[i], g[j], &p[j]))) {
                idx.push_back(j);
                done[j] = 1;
            }
        std::vector<const pat_geometry*> gg;
        std::vector<const float*> ff;
        std::vector<pat_params> pp;
        std::vector<float*> uu;
        std::vector<pat_info> ii(idx.size());
        for (int j : idx) {
            gg.push_back(g[j]);
            ff.push_back(f_dev[j]);
            pp.push_back(p[j]);
            uu.push_back(u_dev[j]);
        }
        int rc = p[i].reg == PAT_WAV ? run_wavelet((int)idx.size(), gg.data(), ff.data(), pp.data(), uu.data(),
                                                   ii.data(), (cudaStream_t)stream, "pat_reconstruct_batched")
                                     : run_batch((int)idx.size(), gg.data(), ff.data(), pp.data(), uu.data(), ii.data(),
                                                 (cudaStream_t)stream, "pat_reconstruct_batched");
        if (infos)
            for (size_t k = 0; k < idx.size(); ++k) infos[idx[k]] = ii[k];
        if (rc) return rc;
    }
    return PAT_OK;
}

// Probe-based choice of the primal-dual balance: every (problem, candidate s) pair runs
// probe_iters iterations from the problem's start, all as one lockstep batch, and for each
// problem the candidate with the smallest relative gap wins.  The probes' images go to
// scratch; nothing else is written.
static int tune_impl(int count, const pat_geometry* const* g, const float* const* f, const pat_params* p,
                     const double* cand, int n_cand, int probe_iters, double* best, double* gaps, cudaStream_t st,
                     const char* who) {
    if (count <= 0 || !g || !f || !p || !cand || !best || n_cand <= 0 || n_cand > 64 || probe_iters <= 0)
        return fail(PAT_ERR_INVALID_ARG, std::string(who) + ": NULL argument, 1..64 candidates and probe_iters > 0");
    for (int i = 0; i < n_cand; ++i)
        if (!(cand[i] > 0) || !std::isfinite(cand[i]))
            return fail(PAT_ERR_INVALID_ARG, std::string(who) + ": candidates must be finite and > 0");
    size_t scratch_floats = 0;
    for (int b = 0; b < count; ++b) {
        int rc = validate(g[b], &p[b], who);
        if (rc) return rc;
        if (!f[b]) return fail(PAT_ERR_INVALID_ARG, std::string(who) + ": NULL data");
        scratch_floats += (size_t)g[b]->desc.n * g[b]->desc.n * n_cand;
    }
    bool any_wav = false;
    for (int b = 0; b < count; ++b) any_wav = any_wav || p[b].reg == PAT_WAV;
    if (any_wav) {
        // with wavelet problems in the set, each problem's candidates run as one batch
        for (int b = 0; b < count; ++b) {
            const size_t nn = (size_t)g[b]->desc.n * g[b]->desc.n;
            float* ub = nullptr;
            PAT_CUDA(cudaMallocAsync(&ub, nn * n_cand * sizeof(float), st));
            std::vector<const pat_geometry*> gb(n_cand, g[b]);
            std::vector<const float*> fb(n_cand, f[b]);
            std::vector<pat_params> qb(n_cand, p[b]);
            std::vector<float*> ubs(n_cand);
            std::vector<pat_info> ii(n_cand);
            for (int c = 0; c < n_cand; ++c) {
                pat_params& q = qb[c];
                q.step_ratio = cand[c];
                q.adapt = PAT_ADAPT_NONE;
                q.iters = probe_iters;
                q.tol = 0.0;
                q.gap_every = 0;
                q.x_out_dev = q.xbar_out_dev = q.y_out_dev = q.x_lo_out_dev = nullptr;
                ubs[c] = ub + nn * c;
            }
            const int rc = p[b].reg == PAT_WAV
                               ? run_wavelet(n_cand, gb.data(), fb.data(), qb.data(), ubs.data(), ii.data(), st, who)
                               : run_batch(n_cand, gb.data(), fb.data(), qb.data(), ubs.data(), ii.data(), st, who);
            cudaFreeAsync(ub, st);
            if (rc) return rc;
            int bi = 0;
            for (int c = 0; c < n_cand; ++c) {
                if (gaps) gaps[b * n_cand + c] = ii[c].rel_gap;
                if (ii[c].rel_gap < ii[bi].rel_gap) bi = c;
            }
            best[b] = cand[bi];
        }
        return PAT_OK;
    }
    float* scratch = nullptr;
    PAT_CUDA(cudaMallocAsync(&scratch, scratch_floats * sizeof(float), st));
    const int B = count * n_cand;
    std::vector<const pat_geometry*> gg(B);
    std::vector<const float*> ff(B);
    std::vector<pat_params> pp(B);
    std::vector<float*> uu(B);
    std::vector<pat_info> ii(B);
    size_t off = 0;
    for (int b = 0; b < count; ++b)
        for (int c = 0; c < n_cand; ++c) {
            const int k = b * n_cand + c;
            gg[k] = g[b];
            ff[k] = f[b];
            pp[k] = p[b];
            pp[k].step_ratio = cand[c];
            pp[k].adapt = PAT_ADAPT_NONE;
            pp[k].iters = probe_iters;
            pp[k].tol = 0.0;
            pp[k].gap_every = 0;
            pp[k].x_out_dev = pp[k].xbar_out_dev = pp[k].y_out_dev = pp[k].x_lo_out_dev = nullptr;
            uu[k] = scratch + off;
            off += (size_t)g[b]->desc.n * g[b]->desc.n;
        }
    int rc = run_batch(B, gg.data(), ff.data(), pp.data(), uu.data(), ii.data(), st, who);
    cudaFreeAsync(scratch, st);
    if (rc) return rc;
    for (int b = 0; b < count; ++b) {
        int bi = 0;
        for (int c = 0; c < n_cand; ++c) {
            const double gc = ii[b * n_cand + c].rel_gap;
            if (gaps) gaps[b * n_cand + c] = gc;
            if (gc < ii[b * n_cand + bi].rel_gap) bi = c;
        }
        best[b] = cand[bi];
    }
    return PAT_OK;
}

extern "C" int pat_tune_step_ratio(const pat_geometry* g, const float* f_dev, const pat_params* p,
                                   const double* candidates_host, int n_candidates, int probe_iters,
                                   double* best_host, double* rel_gaps_host, void* stream) {
    return tune_impl(1, &g, &f_dev, p, candidates_host, n_candidates, probe_iters, best_host, rel_gaps_host,
                     (cudaStream_t)stream, "pat_tune_step_ratio");
}

extern "C" int pat_tune_step_ratio_batched(int count, const pat_geometry* const* g, const float* const* f_dev,
                                           const pat_params* p, const double* candidates_host, int n_candidates,
                                           int probe_iters, double* best_host, double* rel_gaps_host,
                                           void* stream) {
    return tune_impl(count, g, f_dev, p, candidates_host, n_candidates, probe_iters, best_host, rel_gaps_host,
                     (cudaStream_t)stream, "pat_tune_step_ratio_batched");
}

extern "C" int pat_time_phases(int count, const pat_geometry* const* g, const float* const* f_dev,
                               const pat_params* p, int reps, double* us_host, void* stream) {
    if (count < 1 || !g || !f_dev || !p || !us_host || reps < 1 || reps > 100000)
        return fail(PAT_ERR_INVALID_ARG, "pat_time_phases: bad count, pointer or reps");
    if (prof_on()) return fail(PAT_ERR_INVALID_ARG, "pat_time_phases: turn the per-launch profiler off first");
    for (int b = 0; b < count; ++b) {
        const int rc = validate(g[b], &p[b], "pat_time_phases");
        if (rc) return rc;
        if (!f_dev[b]) return fail(PAT_ERR_INVALID_ARG, "pat_time_phases: NULL data");
        if (p[b].reg == PAT_WAV) return fail(PAT_ERR_INVALID_ARG, "pat_time_phases: PAT_WAV has no batch engine");
        if (p[b].iters != p[0].iters || p[b].gap_every != p[0].gap_every)
            return fail(PAT_ERR_INVALID_ARG, "pat_time_phases: a batch needs equal iters and gap_every");
    }
    return time_phases(count, g, f_dev, p, reps, us_host, (cudaStream_t)stream, "pat_time_phases");
}

extern "C" int pat_tune_shapes(int count, pat_geometry* const* g, const float* const* f_dev, const pat_params* p,
                               int reps, const char* cache_path, pat_shapes* chosen_host, void* stream) {
    if (count < 1 || !g || !f_dev || !p || reps < 1 || reps > 100000)
        return fail(PAT_ERR_INVALID_ARG, "pat_tune_shapes: bad count, pointer or reps");
    if (prof_on()) return fail(PAT_ERR_INVALID_ARG, "pat_tune_shapes: turn the per-launch profiler off first");
    for (int b = 0; b < count; ++b) {
        const int rc = validate(g[b], &p[b], "pat_tune_shapes");
        if (rc) return rc;
        if (!f_dev[b]) return fail(PAT_ERR_INVALID_ARG, "pat_tune_shapes: NULL data");
        if (p[b].reg == PAT_WAV) return fail(PAT_ERR_INVALID_ARG, "pat_tune_shapes: PAT_WAV has no batch engine");
    }
    std::vector<ShapeEntry> cache = read_shape_cache(cache_path);
    bool dirty = false;
    for (int b = 0; b < count; ++b) {
        const std::string key = shape_key(g[b], p[b].reg);
        auto it = std::find_if(cache.begin(), cache.end(), [&](const ShapeEntry& e) { return e.key == key; });
        int rc;
        if (it != cache.end()) {
            rc = pat_geometry_set_shapes(g[b], &it->s);
        } else {
            ShapeEntry se;
            se.key = key;
            rc = tune_one(g[b], f_dev[b], &p[b], reps, (cudaStream_t)stream, se);
            if (!rc) {
                cache.push_back(se);
                dirty = true;
            }
        }
        if (rc) return rc;
        if (chosen_host) chosen_host[b] = g[b]->shapes;
    }
    if (cache_path && dirty) return write_shape_cache(cache_path, cache);
    return PAT_OK;
}

extern "C" int pat_steps(const pat_geometry* g, const pat_params* p, float* sig_q_dev, float* tau_u_dev,
                         float* sig_r_dev, float* sig_s_dev, float* tau_v_dev, void* stream) {
    int rc = validate(g, p, "pat_steps");
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->reg == PAT_WAV) {
        WavModel wm;
        if (int mrc = wav_model(g, p, wm)) return mrc;
        return wav_steps(g, wm, sig_q_dev, tau_u_dev, sig_r_dev, step_ratio_of(p), st);
    }
    const int N = g->desc.n;
    const long long NN = (long long)N * N, S = (long long)g->desc.n_det * g->desc.n_t;
    if (p->precond == PAT_PRECOND_SCALAR2) {
        ScalarSteps sc;
        rc = scalar2_steps(g, p, sc, st);
        if (rc) return rc;
        std::vector<float> h;
        auto fill = [&](float* dst, long long n, float v) -> int {
            if (!dst) return PAT_OK;
            h.assign((size_t)n, v);
            PAT_CUDA(cudaMemcpyAsync(dst, h.data(), n * 4, cudaMemcpyHostToDevice, st));
            PAT_CUDA(cudaStreamSynchronize(st));
            return PAT_OK;
        };
        const double s = step_ratio_of(p);
        if ((rc = fill(sig_q_dev, S, (float)(sc.sig_q / s)))) return rc;
        if ((rc = fill(tau_u_dev, NN, (float)(sc.tau * s)))) return rc;
        if ((rc = fill(sig_r_dev, NN, (float)(sc.sig2 / s)))) return rc;
        if (p->reg == PAT_TGV) {
            if ((rc = fill(sig_s_dev, NN, (float)(sc.sig2 / s)))) return rc;
            if ((rc = fill(tau_v_dev, 2 * NN, (float)(sc.tau * s)))) return rc;
        }
        return PAT_OK;
    }
    rc = ensure_precond(g, st);
    if (rc) return rc;
    if (sig_q_dev) {
        k_sig_q<<<ceil_div(S, 256), 256, 0, st>>>(g->pc.krow, sig_q_dev, S);
        PAT_LAUNCH_CHECK("k_sig_q");
    }
    StepArgs sa{N, p->reg, p->gamma, g->pc.kcol, p->xi_dev, tau_u_dev, sig_r_dev,
                p->reg == PAT_TGV ? sig_s_dev : nullptr, p->reg == PAT_TGV ? tau_v_dev : nullptr};
    dim3 blk(32, 8), grd(ceil_div(N, 32), ceil_div(N, 8));
    k_steps_pixels<<<grd, blk, 0, st>>>(sa);
    PAT_LAUNCH_CHECK("k_steps_pixels");
    const double s = step_ratio_of(p);
    if (s != 1.0) {
        auto scale = [&](float* a, long long n, double m) -> int {
            if (!a) return PAT_OK;
            k_scale_f32<<<ceil_div(n, 256), 256, 0, st>>>(a, n, (float)m);
            PAT_LAUNCH_CHECK("k_scale_f32");
            return PAT_OK;
        };
        if ((rc = scale(sig_q_dev, S, 1.0 / s))) return rc;
        if ((rc = scale(tau_u_dev, NN, s))) return rc;
        if ((rc = scale(sig_r_dev, NN, 1.0 / s))) return rc;
        if (p->reg == PAT_TGV) {
            if ((rc = scale(sig_s_dev, NN, 1.0 / s))) return rc;
            if ((rc = scale(tau_v_dev, 2 * NN, s))) return rc;
        }
    }
    return PAT_OK;
}

static int gap_impl(const pat_geometry* g, const float* f, const pat_params* p, const float* x, const float* y,
                    double* out4, cudaStream_t st) {
    Prob pr;
    pr.g = g;
    pr.f = f;
    pr.p = *p;
    pr.p.tol = 0;
    pr.p.adapt = PAT_ADAPT_NONE;
    int rc = alloc_workspace(g, p->reg, pr.ws, st);
    if (rc) return rc;
    const long long S = (long long)g->desc.n_det * g->desc.n_t;
    const int N = g->desc.n;
    InfoDev h{};
    rc = ensure_precond(g, st);
    if (!rc) rc = cudaMemsetAsync(pr.ws.info, 0, sizeof(InfoDev), st) ? PAT_ERR_CUDA : 0;
    if (!rc) rc = cudaMemsetAsync(pr.ws.kt[0], 0, (size_t)N * N * sizeof(int), st) ? PAT_ERR_CUDA : 0;
    if (!rc) rc = launch_absmax(y, S, &pr.ws.info->qmax_bits[0], st);
    std::vector<char> host;
    void* dev = nullptr;
    if (!rc) {
        // one problem, one gap evaluation of (x, y): K^T q then the three gap passes
        GapPlan gp;
        Arena ar(host);
        build_gap_plan(&pr, 1, ar, gp);
        AdjArgs aa = make_adj_args(g, y, nullptr, &pr.ws.info->qmax_bits[0], pr.ws.kt[0], nullptr);
        const size_t adj_off = ar.put(&aa, 1);
        std::vector<int2> amap(g->adj_items);
        for (int i = 0; i < g->adj_items; ++i) amap[i] = make_int2(0, i);
        const size_t amap_off = ar.put(amap.data(), amap.size());
        FwdArgs fa = make_fwd_args(g, x);
        fa.q = const_cast<float*>(y);   // read only by the gap epilogue
        fa.f = f;
        fa.partials = pr.ws.data_part;
        const size_t fa_off = ar.put(&fa, 1);
        GapArgs ga = make_gap_args(pr, kt_view(g, pr.ws.kt[0], &pr.ws.info->qmax_bits[0]), x, nullptr, y + S);
        const size_t ga_off = ar.put(&ga, 1);
        FinalArgs fi = make_final_args(pr);
        const size_t fi_off = ar.put(&fi, 1);
        rc = ar.upload(&dev, st);
        if (!rc) {
            char* b = (char*)dev;
            rc = launch_adjoint_b((const AdjArgs*)(b + adj_off), (const int2*)(b + amap_off), g->adj_items, false, st);
            if (!rc)
                rc = launch_gap_phase((const FwdArgs*)(b + fa_off), (const GapArgs*)(b + ga_off),
                                      (const FinalArgs*)(b + fi_off), gp, b, st);
        }
    }
    if (!rc) rc = cudaMemcpyAsync(&h, pr.ws.info, sizeof(InfoDev), cudaMemcpyDeviceToHost, st) ? PAT_ERR_CUDA : 0;
    if (dev) cudaFreeAsync(dev, st);
    cudaFreeAsync(pr.ws.base, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (!rc && se != cudaSuccess) rc = cuda_fail(se, "pat_duality_gap");
    if (rc) return rc;
    out4[0] = h.primal;
    out4[1] = h.dual;
    out4[2] = h.gap;
    out4[3] = h.rel_gap;
    return PAT_OK;
}

extern "C" int pat_duality_gap(const pat_geometry* g, const float* f_dev, const pat_params* p, const float* x_dev,
                               const float* y_dev, double* out4_host, void* stream) {
    if (p && p->reg == PAT_WAV)
        return fail(PAT_ERR_INVALID_ARG, "pat_duality_gap: not available for PAT_WAV (pat_reconstruct reports its gap)");
    int rc = validate(g, p, "pat_duality_gap");
    if (rc) return rc;
    if (!f_dev || !x_dev || !y_dev || !out4_host) return fail(PAT_ERR_INVALID_ARG, "pat_duality_gap: NULL argument");
    return gap_impl(g, f_dev, p, x_dev, y_dev, out4_host, (cudaStream_t)stream);
}

__global__ void k_direction_field(int N, const float* __restrict__ w, float eta, float* __restrict__ xi) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= N || gy >= N) return;
    const int gi = gy * N + gx;
    const float g0 = gx < N - 1 ? w[gi + 1] - w[gi] : 0.f;
    const float g1 = gy < N - 1 ? w[gi + N] - w[gi] : 0.f;
    const float inv = rsqrtf(g0 * g0 + g1 * g1 + eta * eta);
    xi[gi] = g0 * inv;
    xi[(size_t)N * N + gi] = g1 * inv;
}

extern "C" int pat_direction_field(int n, const float* w_dev, double eta, float* xi_dev, void* stream) {
    if (n < 2 || !w_dev || !xi_dev) return fail(PAT_ERR_INVALID_ARG, "pat_direction_field: bad argument");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(PAT_ERR_INVALID_ARG, "pat_direction_field: eta must be > 0");
    dim3 blk(32, 8), grd(ceil_div(n, 32), ceil_div(n, 8));
    k_direction_field<<<grd, blk, 0, (cudaStream_t)stream>>>(n, w_dev, (float)eta, xi_dev);
    PAT_LAUNCH_CHECK("k_direction_field");
    return PAT_OK;
}
