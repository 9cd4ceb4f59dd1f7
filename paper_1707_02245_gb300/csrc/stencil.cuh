// Finite-difference conventions and pointwise maps of the PDHG iteration (device side).
//
// Gradient (Sec. 2.1, "matrix versions" of Sec. 3.3.1): forward differences with unit
// spacing and a zero difference on the last column / row.  div = -grad^T.
// Symmetrised gradient E v = (d_x^- v1, d_y^- v2, (d_y^- v1 + d_x^- v2)/sqrt 2) with the
// backward difference d^- = -(d^+)^T; the third component is the off-diagonal entry in
// orthonormal coordinates so the Frobenius norm is the Euclidean norm of the three.
// Both backward differences and div read a field "masked" to zero on the last index:
//   (d^- v)(i) = v'(i) - v'(i-1),  v'(i) = v(i) for 0 <= i < N-1, else 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace pat {

constexpr float kInvSqrt2f = 0.70710678118654752f;
constexpr double kSqrt2 = 1.4142135623730951;

// radius * p / max(radius, |p|) for a 2- or 3-vector (Sec. 3.2).  Inside the ball p is
// kept as it is; outside, the scale radius / |p| comes from one reciprocal square root
// (a relative error of a few 1e-7, far inside the FP32 iterates' own).  With radius 0 the
// result is 0.
// Projections onto the balls of the pointwise dual constraints (Sec. 3.2).  Every rounding
// is spelled out (no contraction into fused multiply-adds), so that each kernel, and each
// unrolled copy within a kernel, that inlines them computes the same bits.
__device__ __forceinline__ void proj2(float& a, float& b, float radius) {
    const float n2 = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
    const float sc = n2 > __fmul_rn(radius, radius) ? __fmul_rn(radius, rsqrtf(n2)) : 1.f;
    a = __fmul_rn(a, sc);
    b = __fmul_rn(b, sc);
}

__device__ __forceinline__ void proj3(float& a, float& b, float& c, float radius) {
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
    const float sc = n2 > __fmul_rn(radius, radius) ? __fmul_rn(radius, rsqrtf(n2)) : 1.f;
    a = __fmul_rn(a, sc);
    b = __fmul_rn(b, sc);
    c = __fmul_rn(c, sc);
}

// Inline diagonal steps of the Pock-Chambolle rule (alpha = 1) for the stencil rows.
// a = [i < N-1], b = [j < N-1], ex = [i < N-1] + [i >= 1], ey likewise.
// TV  r rows: |d_x^+| row sum 2a, |d_y^+| 2b; the group takes 1/max (1 if both vanish).
// TGV r rows add the -I entry: 2a + 1, 2b + 1.
// TGV s rows: ex, ey, (ex + ey)/sqrt 2.   v columns: 1 + 2a + sqrt2 b, 1 + 2b + sqrt2 a.
// Each takes a few values only, so the reciprocals are constants folded at compile time
// (the same IEEE quotients a run-time division gives) picked by the pixel's edge flags.
__device__ __forceinline__ float sig_r_tv(int i, int j, int N) {
    return ((i < N - 1) || (j < N - 1)) ? 0.5f : 1.f;   // 1 / max(2a, 2b); 1 if both vanish
}
__device__ __forceinline__ float sig_r_tgv(int i, int j, int N) {
    return ((i < N - 1) || (j < N - 1)) ? 1.f / 3.f : 1.f;   // 1 / max(2a + 1, 2b + 1)
}
constexpr float cmaxf(float x, float y) { return x > y ? x : y; }
constexpr float sig_s_entry(float ex, float ey) { return 1.f / cmaxf(cmaxf(ex, ey), (ex + ey) * kInvSqrt2f); }
constexpr float tau_v_entry(float a, float b) { return 1.f / (1.f + 2.f * a + 1.41421356237f * b); }
__device__ __forceinline__ float sig_s_tgv(int i, int j, int N) {
    // 1 / max(max(ex, ey), (ex + ey) / sqrt 2); with N >= 2 every pixel has ex, ey in {1, 2}
    const bool x2 = (i < N - 1) && (i >= 1), y2 = (j < N - 1) && (j >= 1);
    constexpr float t11 = sig_s_entry(1.f, 1.f), t12 = sig_s_entry(1.f, 2.f), t21 = sig_s_entry(2.f, 1.f),
                    t22 = sig_s_entry(2.f, 2.f);
    return x2 ? (y2 ? t22 : t21) : (y2 ? t12 : t11);
}
__device__ __forceinline__ float tau_v1_tgv(int i, int j, int N) {
    // 1 / (1 + 2a + sqrt2 b)
    constexpr float t00 = tau_v_entry(0.f, 0.f), t01 = tau_v_entry(0.f, 1.f), t10 = tau_v_entry(1.f, 0.f),
                    t11 = tau_v_entry(1.f, 1.f);
    const bool a = i < N - 1, b = j < N - 1;
    return a ? (b ? t11 : t10) : (b ? t01 : t00);
}
__device__ __forceinline__ float tau_v2_tgv(int i, int j, int N) {
    // 1 / (1 + 2b + sqrt2 a)
    constexpr float t00 = tau_v_entry(0.f, 0.f), t01 = tau_v_entry(0.f, 1.f), t10 = tau_v_entry(1.f, 0.f),
                    t11 = tau_v_entry(1.f, 1.f);
    const bool a = i < N - 1, b = j < N - 1;
    return b ? (a ? t11 : t10) : (a ? t01 : t00);
}

// (hi, lo) += delta by an error-free TwoSum followed by renormalisation: the pair holds
// hi + lo to about 48 significant bits, so primal updates far below ulp(hi) keep
// accumulating instead of rounding away (the FP32 iterates would otherwise stall once
// tau |K^T q - div r| drops below half an ulp of u).
__device__ __forceinline__ void add_compensated(float& hi, float& lo, float delta) {
    const float s = __fadd_rn(hi, delta);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(delta, bb));
    const float t = __fadd_rn(lo, e);
    const float h2 = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(h2, s));
    hi = h2;
}

// The low word of a compensated pair is stored in 16 bits as a bfloat16 (round to nearest
// even): 8 significant bits of a word below half an ulp of the high word, so the pair
// holds hi + lo to about 32 significant bits, and the conversions are single
// instructions.  lo_round returns the stored value of lo.
__device__ __forceinline__ unsigned short lo_encode(float lo) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(lo));
}
__device__ __forceinline__ float lo_decode(unsigned short q) { return __bfloat162float(__ushort_as_bfloat16(q)); }
__device__ __forceinline__ float lo_round(float lo) { return lo_decode(lo_encode(lo)); }

// D_xi = I - gamma xi xi^T applied to p (symmetric).  The roundings are spelled out so
// that every kernel that inlines this computes the same bits.
__device__ __forceinline__ void dxi_apply(float xi0, float xi1, float gamma, float p0, float p1, float& o0,
                                          float& o1) {
    const float dot = __fmaf_rn(xi0, p0, __fmul_rn(xi1, p1));
    const float gd = __fmul_rn(gamma, dot);
    o0 = __fmaf_rn(-xi0, gd, p0);
    o1 = __fmaf_rn(-xi1, gd, p1);
}

}  // namespace pat
