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
#include <cuda_runtime.h>

namespace pat {

constexpr float kInvSqrt2f = 0.70710678118654752f;
constexpr double kSqrt2 = 1.4142135623730951;

// radius * p / max(radius, |p|) for a 2- or 3-vector (Sec. 3.2); 0 when both are 0.
__device__ __forceinline__ void proj2(float& a, float& b, float radius) {
    const float den = fmaxf(radius, sqrtf(a * a + b * b));
    const float sc = den > 0.f ? radius / den : 0.f;
    a *= sc;
    b *= sc;
}

__device__ __forceinline__ void proj3(float& a, float& b, float& c, float radius) {
    const float den = fmaxf(radius, sqrtf(a * a + b * b + c * c));
    const float sc = den > 0.f ? radius / den : 0.f;
    a *= sc;
    b *= sc;
    c *= sc;
}

// Inline diagonal steps of the Pock-Chambolle rule (alpha = 1) for the stencil rows.
// a = [i < N-1], b = [j < N-1], ex = [i < N-1] + [i >= 1], ey likewise.
// TV  r rows: |d_x^+| row sum 2a, |d_y^+| 2b; the group takes 1/max (1 if both vanish).
// TGV r rows add the -I entry: 2a + 1, 2b + 1.
// TGV s rows: ex, ey, (ex + ey)/sqrt 2.   v columns: 1 + 2a + sqrt2 b, 1 + 2b + sqrt2 a.
__device__ __forceinline__ float sig_r_tv(int i, int j, int N) {
    const float m = fmaxf(2.f * (i < N - 1), 2.f * (j < N - 1));
    return m > 0.f ? 1.f / m : 1.f;
}
__device__ __forceinline__ float sig_r_tgv(int i, int j, int N) {
    return 1.f / fmaxf(2.f * (i < N - 1) + 1.f, 2.f * (j < N - 1) + 1.f);
}
__device__ __forceinline__ float sig_s_tgv(int i, int j, int N) {
    const float ex = (float)((i < N - 1) + (i >= 1)), ey = (float)((j < N - 1) + (j >= 1));
    return 1.f / fmaxf(fmaxf(ex, ey), (ex + ey) * kInvSqrt2f);
}
__device__ __forceinline__ float tau_v1_tgv(int i, int j, int N) {
    return 1.f / (1.f + 2.f * (i < N - 1) + 1.41421356237f * (j < N - 1));
}
__device__ __forceinline__ float tau_v2_tgv(int i, int j, int N) {
    return 1.f / (1.f + 2.f * (j < N - 1) + 1.41421356237f * (i < N - 1));
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

// D_xi = I - gamma xi xi^T applied to p (symmetric).
__device__ __forceinline__ void dxi_apply(float xi0, float xi1, float gamma, float p0, float p1, float& o0,
                                          float& o1) {
    const float dot = xi0 * p0 + xi1 * p1;
    o0 = p0 - gamma * xi0 * dot;
    o1 = p1 - gamma * xi1 * dot;
}

}  // namespace pat
