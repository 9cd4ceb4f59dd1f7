"""Plain FP64 CPU oracle for the dual-tree complex wavelet transform (DT-CWT) of the
wavelet model of Sec. 2.2 (eq. (min_wav)): min_u 1/2 ||Ku - f||^2 + alpha ||W u||_1 with W
the 2-D dual-tree complex wavelet transform.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module.  The CUDA library never imports,
links or executes it, and it shares no code, tables or helpers with the CUDA path.

The transform (Kingsbury's dual tree, Sec. 2.2; the paper uses the Cai-Li / Selesnick
implementation of it, footnote of Sec. 3.3.1):
- Two real filter banks, tree a and tree b, each an orthonormal two-channel bank, so each
  separable 2-D transform below is orthonormal.
- Level 1: the same filters in both trees, tree b delayed by one sample (its input index
  is offset by one), i.e. half a sample at the rate of the level-1 coefficients.
- Levels >= 2: "Q-shift" filters: tree b's low-pass filter is tree a's reversed in time,
  and tree a's has its centre a quarter sample before its midpoint, so that the trees'
  scaling functions are half a sample apart at every level.
- 2-D: four separable transforms (x tree, y tree) in {a, b}^2, index t = 2 p + q with p the
  tree along x and q along y: aa, ab, ba, bb.  Each has J levels in the Mallat layout of an
  N x N array (level l splits the top-left M x M block, M = N / 2^(l-1), into LL, HL
  (high-pass along x), LH (high-pass along y) and HH).
- W u = (1/2) [T_aa u; T_ab u; T_ba u; T_bb u] followed, at every detail position, by
  the orthogonal change to two complex coefficients
      z1 = ((aa - bb) + i (ab + ba)) / sqrt 2,   z2 = ((aa + bb) + i (ba - ab)) / sqrt 2,
  stored as four real planes (Re z1, Im z1, Re z2, Im z2).  At the LL positions of the
  last level the four planes hold (1/2) the four trees' LL coefficients.  Each tree is
  orthonormal and the change is orthogonal, so W^T W = I: W is a tight frame with
  ||W|| = 1 and W^-1 = W^T (the property Sec. 3.3.1 uses).
- ||W u||_1 is the sum of the moduli of the complex detail coefficients plus the absolute
  values of the LL coefficients.  Its dual prox (Sec. 3.2) projects every complex
  coefficient onto the disc of radius alpha and clips every LL coefficient to
  [-alpha, alpha].

Readings (filters): Kingsbury's published filter coefficients are not available here, so
the default filters are closed forms with the properties the construction asks for:
- level 1: Daubechies' orthonormal 4-tap filter (1+s3, 3+s3, 3-s3, 1-s3)/(4 sqrt 2);
- levels >= 2: the orthonormal 4-tap filter of the one-angle lattice with sin(theta) =
  1/4, h = (5 - s15, 5 + s15, 3 + s15, 3 - s15) / (8 sqrt 2) (s15 = sqrt 15), whose centre
  sum_n n h[n] / sum_n h[n] is 1.25, a quarter sample before the midpoint 1.5;
- high-pass g[n] = (-1)^n h[L - 1 - n].
Any orthonormal pair can be passed instead (the construction does not depend on the
values).  One analysis step along an axis of length M with filter (h, g) and offset o:
  a[k] = sum_n h[n] x[(2k + n + o) mod M],  d[k] = sum_n g[n] x[(2k + n + o) mod M].
Periodic extension; N divisible by 2^J.

Pins: tests/test_dtcwt_oracle_pins.py.
"""
from __future__ import annotations

import math

import numpy as np

S3 = math.sqrt(3.0)
S15 = math.sqrt(15.0)
D4 = np.array([1 + S3, 3 + S3, 3 - S3, 1 - S3]) / (4 * math.sqrt(2.0))
QSHIFT4 = np.array([5 - S15, 5 + S15, 3 + S15, 3 - S15]) / (8 * math.sqrt(2.0))
TREES = ("aa", "ab", "ba", "bb")   # t = 2 p + q: p the tree along x, q along y


def highpass(h) -> np.ndarray:
    """g[n] = (-1)^n h[L - 1 - n], the orthonormal partner of h."""
    h = np.asarray(h, dtype=np.float64)
    L = h.size
    return np.array([(-1) ** n * h[L - 1 - n] for n in range(L)])


def default_filters():
    """(level-1 low-pass, Q-shift low-pass of tree a) of the default bank."""
    return D4.copy(), QSHIFT4.copy()


def _axis_filters(tree: int, level: int, filters):
    """(h, g, offset) of one tree (0 = a, 1 = b) at one level (1-based)."""
    h1, hq = (np.asarray(f, dtype=np.float64) for f in filters)
    if level == 1:
        return h1, highpass(h1), tree
    h = hq if tree == 0 else hq[::-1].copy()
    return h, highpass(h), 0


def _analyse_axis(x, axis, h, g, off):
    """One analysis step along ``axis``: returns (low, high) halves."""
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    M = x.shape[-1]
    L = len(h)
    idx = (2 * np.arange(M // 2)[:, None] + np.arange(L)[None, :] + off) % M
    seg = x[..., idx]
    return np.moveaxis(seg @ h, -1, axis), np.moveaxis(seg @ g, -1, axis)


def _synthesise_axis(lo, hi, axis, h, g, off):
    """Transpose of ``_analyse_axis``: x[m] = sum over (k, n) with m = 2k + n + o (mod M)
    of h[n] lo[k] + g[n] hi[k]."""
    lo = np.moveaxis(np.asarray(lo, dtype=np.float64), axis, -1)
    hi = np.moveaxis(np.asarray(hi, dtype=np.float64), axis, -1)
    half = lo.shape[-1]
    M = 2 * half
    x = np.zeros(lo.shape[:-1] + (M,))
    for n in range(len(h)):
        pos = (2 * np.arange(half) + n + off) % M
        np.add.at(x, (Ellipsis, pos), h[n] * lo + g[n] * hi)
    return np.moveaxis(x, -1, axis)


def tree_transform(u, levels: int, t: int, filters=None) -> np.ndarray:
    """T_t u: the separable orthonormal transform of tree t (x tree p = t // 2, y tree
    q = t % 2) in the Mallat layout."""
    filters = default_filters() if filters is None else filters
    c = np.array(u, dtype=np.float64)
    N = c.shape[0]
    if c.shape != (N, N) or N % (1 << levels):
        raise ValueError("image must be N x N with N divisible by 2^levels")
    p, q = t // 2, t % 2
    M = N
    for lev in range(1, levels + 1):
        hx, gx, ox = _axis_filters(p, lev, filters)
        hy, gy, oy = _axis_filters(q, lev, filters)
        blk = c[:M, :M]
        lo_y, hi_y = _analyse_axis(blk, 0, hy, gy, oy)
        ll, hl = _analyse_axis(lo_y, 1, hx, gx, ox)
        lh, hh = _analyse_axis(hi_y, 1, hx, gx, ox)
        h2 = M // 2
        c[:h2, :h2], c[:h2, h2:M], c[h2:M, :h2], c[h2:M, h2:M] = ll, hl, lh, hh
        M = h2
    return c


def tree_transpose(c, levels: int, t: int, filters=None) -> np.ndarray:
    """T_t^T c (= T_t^-1 c)."""
    filters = default_filters() if filters is None else filters
    u = np.array(c, dtype=np.float64)
    N = u.shape[0]
    p, q = t // 2, t % 2
    M = N >> (levels - 1)
    for lev in range(levels, 0, -1):
        hx, gx, ox = _axis_filters(p, lev, filters)
        hy, gy, oy = _axis_filters(q, lev, filters)
        h2 = M // 2
        ll, hl, lh, hh = u[:h2, :h2], u[:h2, h2:M], u[h2:M, :h2], u[h2:M, h2:M]
        lo_y = _synthesise_axis(ll, hl, 1, hx, gx, ox)
        hi_y = _synthesise_axis(lh, hh, 1, hx, gx, ox)
        u[:M, :M] = _synthesise_axis(lo_y, hi_y, 0, hy, gy, oy)
        M *= 2
    return u


def ll_mask(n: int, levels: int) -> np.ndarray:
    """True at the LL positions of the last level (the top-left (n / 2^J)^2 block)."""
    m = np.zeros((n, n), dtype=bool)
    s = n >> levels
    m[:s, :s] = True
    return m


def combine(T) -> np.ndarray:
    """The four (1/2-scaled) tree arrays (aa, ab, ba, bb) -> the four real planes of W u."""
    aa, ab, ba, bb = (np.asarray(x, dtype=np.float64) for x in T)
    r2 = math.sqrt(2.0)
    return np.stack([(aa - bb) / r2, (ab + ba) / r2, (aa + bb) / r2, (ba - ab) / r2])


def uncombine(C) -> np.ndarray:
    """Transpose (= inverse) of ``combine``."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.float64) for x in C)
    r2 = math.sqrt(2.0)
    return np.stack([(c0 + c2) / r2, (c1 - c3) / r2, (c1 + c3) / r2, (c2 - c0) / r2])


def dtcwt2(u, levels: int, filters=None) -> np.ndarray:
    """W u as a (4, N, N) array: complex detail coefficients as (Re z1, Im z1, Re z2, Im z2)
    planes, and at the last level's LL positions the four trees' LL coefficients."""
    u = np.asarray(u, dtype=np.float64)
    T = np.stack([0.5 * tree_transform(u, levels, t, filters) for t in range(4)])
    C = combine(T)
    m = ll_mask(u.shape[0], levels)
    C[:, m] = T[:, m]
    return C


def idtcwt2(C, levels: int, filters=None) -> np.ndarray:
    """W^T C (= W^-1 C)."""
    C = np.asarray(C, dtype=np.float64)
    T = uncombine(C)
    m = ll_mask(C.shape[1], levels)
    T[:, m] = C[:, m]
    return sum(0.5 * tree_transpose(T[t], levels, t, filters) for t in range(4))


def l1(C, levels: int) -> float:
    """||W u||_1 of coefficients C: moduli of the complex detail coefficients plus |LL|."""
    C = np.asarray(C, dtype=np.float64)
    m = ll_mask(C.shape[1], levels)
    det = np.hypot(C[0], C[1]) + np.hypot(C[2], C[3])
    return float(det[~m].sum() + np.abs(C[:, m]).sum())


def project(C, alpha: float, levels: int) -> np.ndarray:
    """The dual prox of alpha ||.||_1 (Sec. 3.2): every complex detail coefficient onto the
    disc of radius alpha, every LL coefficient clipped to [-alpha, alpha]."""
    C = np.array(C, dtype=np.float64)
    m = ll_mask(C.shape[1], levels)
    for a, b in ((0, 1), (2, 3)):
        mod = np.hypot(C[a], C[b])
        sc = np.where(mod > alpha, alpha / np.where(mod > 0, mod, 1.0), 1.0)
        sc[m] = 1.0
        C[a] *= sc
        C[b] *= sc
    C[:, m] = np.clip(C[:, m], -alpha, alpha)
    return C


def dense_matrix(n: int, levels: int, filters=None) -> np.ndarray:
    """W as an explicit (4 n^2) x n^2 matrix (columns W e_j), for small n."""
    W = np.zeros((4 * n * n, n * n))
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1.0
        W[:, j] = dtcwt2(e.reshape(n, n), levels, filters).ravel()
    return W


def abs_sums(n: int, levels: int, filters=None):
    """Row sums (per coefficient, (4, n, n)) and column sums (per pixel, (n, n)) of |W|,
    accumulated column by column (no dense matrix is stored)."""
    rows = np.zeros(4 * n * n)
    cols = np.zeros(n * n)
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1.0
        w = np.abs(dtcwt2(e.reshape(n, n), levels, filters).ravel())
        rows += w
        cols[j] = w.sum()
    return rows.reshape(4, n, n), cols.reshape(n, n)


# ---------------------------------------------------------------------------------------
# the DT-CWT model in PDHG (Algorithm 1 with grad -> W, div -> -W^T)
# ---------------------------------------------------------------------------------------

def cwt_steps(kcol, krow, n: int, levels: int, filters=None):
    """Pock-Chambolle diagonal steps (alpha = 1) for A = (K; W): sigma_q = 1 / K 1,
    tau_u = 1 / (K^T 1 + |W|^T 1), and sigma_r = 1 / (|W| 1) per LL coefficient.  The two
    rows of a complex coefficient share one step, 1 / (the larger of their two row sums)
    (reading R5 of pat_oracle: the dual prox of a pointwise disc is the projection onto it
    only when the disc's components share their step); a zero sum gives 1."""
    rows, cols = abs_sums(n, levels, filters)
    m = ll_mask(n, levels)
    grp = rows.copy()
    for a, b in ((0, 1), (2, 3)):
        mx = np.maximum(rows[a], rows[b])
        grp[a] = np.where(m, rows[a], mx)
        grp[b] = np.where(m, rows[b], mx)

    def inv(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where(x > 0, 1.0 / np.where(x > 0, x, 1.0), 1.0)
    return inv(krow), inv(grp), inv(np.asarray(kcol).reshape(n, n) + cols)


def cwt_gap(Kf, KTf, f, n, levels, alpha, u, q, r, box_u=2.0, filters=None, KTq=None):
    """Box-restricted gap (reading R7 of pat_oracle):
    P = 1/2 |Ku - f|^2 + alpha ||W u||_1,  D = -(1/2 |q|^2 + <q, f>) - U |K^T q + W^T r|_1."""
    f = np.asarray(f, dtype=np.float64).ravel()
    res = np.asarray(Kf(u)).ravel() - f
    primal = 0.5 * float(res @ res) + alpha * l1(dtcwt2(u, levels, filters), levels)
    if KTq is None:
        KTq = np.asarray(KTf(q)).reshape(n, n)
    dual = -(0.5 * float(q @ q) + float(q @ f)) - box_u * float(np.sum(np.abs(KTq + idtcwt2(r, levels, filters))))
    gap = primal - dual
    return {"primal": primal, "dual": dual, "gap": gap, "rel_gap": gap / primal if primal > 0 else 0.0}


def pdhg_cwt(Kf, KTf, f, n: int, levels: int, alpha: float, iters: int, sig_q, sig_r, tau_u,
             theta: float = 1.0, box_u: float = 2.0, gap_every: int = 0, step_ratio: float = 1.0, filters=None):
    """Algorithm 1 for eq. (min_wav) with the DT-CWT.  Returns (u, q, r, history)."""
    f = np.asarray(f, dtype=np.float64).ravel()
    sq, sr, tu = sig_q / step_ratio, sig_r / step_ratio, tau_u * step_ratio
    u = np.zeros((n, n))
    ubar = u.copy()
    q = np.zeros(f.size)
    r = np.zeros((4, n, n))
    hist = []
    for it in range(iters):
        q = (q + sq * (np.asarray(Kf(ubar)).ravel() - f)) / (1.0 + sq)               # prox of F1*
        r = project(r + sr * dtcwt2(ubar, levels, filters), alpha, levels)          # prox of F2*
        KTq = np.asarray(KTf(q)).reshape(n, n)
        u_new = u - tu * (KTq + idtcwt2(r, levels, filters))
        ubar = u_new + theta * (u_new - u)
        u = u_new
        done = it + 1
        if (gap_every and done % gap_every == 0) or done == iters:
            g = cwt_gap(Kf, KTf, f, n, levels, alpha, u, q, r, box_u, filters, KTq=KTq)
            hist.append((done, g["gap"], g["rel_gap"]))
    return u, q, r, hist
