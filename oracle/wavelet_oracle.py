"""Plain FP64 CPU oracle for the wavelet-regularised reconstruction of Sec. 2.2
(eq. (min_wav)):  min_u 1/2 ||Ku - f||^2 + alpha ||W u||_1.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module.  The CUDA library never imports,
links or executes it, and it shares no code, tables or helpers with the CUDA path.

Sec. 3 obtains the wavelet model from the TV model (Algorithm 1) by replacing grad with W
and div with W^-1.  W is a tight frame, so W^-1 = W^T.  F2 becomes alpha ||.||_1 of a
scalar field, so its dual prox is the clip to [-alpha, alpha] of every coefficient.

Reading WV1 (the transform): the paper's dual-tree complex wavelet transform needs
Kingsbury's Q-shift filters and the Cai-Li code, neither available here.  W is instead
the orthonormal separable 2-D discrete wavelet transform:
- Daubechies' 4-tap filters (closed form h = (1+s3, 3+s3, 3-s3, 1-s3) / (4 sqrt 2) with
  s3 = sqrt 3, and g[n] = (-1)^n h[3-n]);
- periodic extension and J levels (N divisible by 2^J);
- the Mallat layout: level l splits the top-left (N/2^l)^2 block into LL (top-left), HL
  (top-right: high-pass along x), LH (bottom-left: high-pass along y) and HH.
W is orthonormal (W^T W = I) like the paper's tight frame with ||W|| = 1 (Sec. 3.3.2).

One level along an axis of length M:
  a[k] = sum_n h[n] x[(2k + n) mod M],  d[k] = sum_n g[n] x[(2k + n) mod M].

Pins (tests/test_wavelet_oracle_pins.py): the filters' closed-form properties
(orthonormality of even shifts, two vanishing moments); the dense matrix of W is
orthogonal; perfect reconstruction; ramps have zero detail away from the wrap; the dense
|W| row and column sums against the separable formula the CUDA path uses.
"""
from __future__ import annotations

import math

import numpy as np

S3 = math.sqrt(3.0)
H = np.array([1 + S3, 3 + S3, 3 - S3, 1 - S3]) / (4 * math.sqrt(2.0))
G = np.array([(-1) ** n * H[3 - n] for n in range(4)])


def _analyse_axis(x, axis):
    """One level along ``axis``: returns (low, high) halves."""
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    M = x.shape[-1]
    idx = (2 * np.arange(M // 2)[:, None] + np.arange(4)[None, :]) % M
    seg = x[..., idx]                     # (..., M/2, 4)
    lo = seg @ H
    hi = seg @ G
    return np.moveaxis(lo, -1, axis), np.moveaxis(hi, -1, axis)


def _synthesise_axis(lo, hi, axis):
    """Transpose of ``_analyse_axis``: x[m] = sum_k h[m-2k] lo[k] + g[m-2k] hi[k]."""
    lo = np.moveaxis(np.asarray(lo, dtype=np.float64), axis, -1)
    hi = np.moveaxis(np.asarray(hi, dtype=np.float64), axis, -1)
    half = lo.shape[-1]
    M = 2 * half
    x = np.zeros(lo.shape[:-1] + (M,))
    for n in range(4):
        pos = (2 * np.arange(half) + n) % M
        np.add.at(x, (Ellipsis, pos), H[n] * lo + G[n] * hi)
    return np.moveaxis(x, -1, axis)


def dwt2(u, levels: int):
    """W u in the Mallat layout (N x N); N must be divisible by 2^levels."""
    c = np.array(u, dtype=np.float64)
    N = c.shape[0]
    if c.shape != (N, N) or N % (1 << levels):
        raise ValueError("image must be N x N with N divisible by 2^levels")
    M = N
    for _ in range(levels):
        blk = c[:M, :M]
        lo_y, hi_y = _analyse_axis(blk, 0)            # along y (rows index)
        ll, hl = _analyse_axis(lo_y, 1)               # along x
        lh, hh = _analyse_axis(hi_y, 1)
        h2 = M // 2
        c[:h2, :h2], c[:h2, h2:M], c[h2:M, :h2], c[h2:M, h2:M] = ll, hl, lh, hh
        M = h2
    return c


def idwt2(c, levels: int):
    """W^T c (= W^-1 c)."""
    u = np.array(c, dtype=np.float64)
    N = u.shape[0]
    M = N >> (levels - 1)
    for _ in range(levels):
        h2 = M // 2
        ll, hl, lh, hh = u[:h2, :h2], u[:h2, h2:M], u[h2:M, :h2], u[h2:M, h2:M]
        lo_y = _synthesise_axis(ll, hl, 1)
        hi_y = _synthesise_axis(lh, hh, 1)
        u[:M, :M] = _synthesise_axis(lo_y, hi_y, 0)
        M *= 2
    return u


def dense_matrix(n: int, levels: int) -> np.ndarray:
    """W as an explicit n^2 x n^2 matrix (columns W e_j), for small n."""
    W = np.zeros((n * n, n * n))
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1.0
        W[:, j] = dwt2(e.reshape(n, n), levels).ravel()
    return W


def abs_sums(n: int, levels: int) -> tuple[np.ndarray, np.ndarray]:
    """Row sums (per coefficient, Mallat layout) and column sums (per pixel) of |W|, from
    the dense matrix."""
    A = np.abs(dense_matrix(n, levels))
    return A.sum(axis=1).reshape(n, n), A.sum(axis=0).reshape(n, n)


# ---------------------------------------------------------------------------------------
# the wavelet model in PDHG (Algorithm 1 with grad -> W, div -> -W^T)
# ---------------------------------------------------------------------------------------

def wavelet_steps(kcol, krow, n: int, levels: int):
    """Pock-Chambolle diagonal steps (alpha = 1) for A = (K; W): sigma_q = 1 / K 1,
    sigma_r = 1 / (|W| 1), tau_u = 1 / (K^T 1 + |W|^T 1); a zero sum gives 1."""
    rows, cols = abs_sums(n, levels)

    def inv(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where(x > 0, 1.0 / np.where(x > 0, x, 1.0), 1.0)
    return inv(krow), inv(rows), inv(np.asarray(kcol).reshape(n, n) + cols)


def pdhg_wavelet(Kf, KTf, f, n: int, levels: int, alpha: float, iters: int, sig_q, sig_r, tau_u,
                 theta: float = 1.0, box_u: float = 2.0, gap_every: int = 0, step_ratio: float = 1.0):
    """Algorithm 1 for eq. (min_wav).  Kf, KTf apply K and K^T.  Returns
    (u, q, r, history), history = [(iteration, gap, rel_gap)] at the gap evaluations
    (every gap_every iterations and after the last one)."""
    f = np.asarray(f, dtype=np.float64).ravel()
    sq, sr, tu = sig_q / step_ratio, sig_r / step_ratio, tau_u * step_ratio
    u = np.zeros((n, n))
    ubar = u.copy()
    q = np.zeros(f.size)
    r = np.zeros((n, n))
    hist = []
    for it in range(iters):
        q = (q + sq * (np.asarray(Kf(ubar)).ravel() - f)) / (1.0 + sq)       # prox of F1*
        r = np.clip(r + sr * dwt2(ubar, levels), -alpha, alpha)            # prox of F2*
        KTq = np.asarray(KTf(q)).reshape(n, n)
        u_new = u - tu * (KTq + idwt2(r, levels))
        ubar = u_new + theta * (u_new - u)
        u = u_new
        done = it + 1
        if (gap_every and done % gap_every == 0) or done == iters:
            g = wavelet_gap(Kf, KTf, f, n, levels, alpha, u, q, r, box_u, KTq=KTq)
            hist.append((done, g["gap"], g["rel_gap"]))
    return u, q, r, hist


def wavelet_gap(Kf, KTf, f, n, levels, alpha, u, q, r, box_u=2.0, KTq=None):
    """Box-restricted gap (reading R7 of pat_oracle):
    P = 1/2 |Ku - f|^2 + alpha |W u|_1,  D = -(1/2 |q|^2 + <q, f>) - U |K^T q + W^T r|_1."""
    f = np.asarray(f, dtype=np.float64).ravel()
    res = np.asarray(Kf(u)).ravel() - f
    primal = 0.5 * float(res @ res) + alpha * float(np.sum(np.abs(dwt2(u, levels))))
    if KTq is None:
        KTq = np.asarray(KTf(q)).reshape(n, n)
    dual = -(0.5 * float(q @ q) + float(q @ f)) - box_u * float(np.sum(np.abs(KTq + idwt2(r, levels))))
    gap = primal - dual
    return {"primal": primal, "dual": dual, "gap": gap, "rel_gap": gap / primal if primal > 0 else 0.0}
