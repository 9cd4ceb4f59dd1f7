"""Pins for the FP64 oracle of the wavelet model (oracle/wavelet_oracle.py):

* Daubechies' 4-tap filters: unit norm, orthogonal even shifts, h and g orthogonal, two
  vanishing moments of g, and sum h = sqrt 2 (closed-form properties, not the formula);
* the dense matrix of the multi-level 2-D transform is orthogonal (W^T W = I) and idwt2
  is its transpose;
* a linear ramp has zero detail coefficients away from the periodic wrap;
* a constant image maps to a single LL block of value c 2^J;
* the separable |W| row/column sums (the CUDA path's formula) equal the dense sums;
* the wavelet PDHG reaches its saddle point: the gap of a long run is tiny, and with K = I
  and alpha -> infinity the solution is the constant image that W keeps in LL.
"""
import math

import numpy as np
import pytest

from oracle import wavelet_oracle as WO


def test_filter_closed_form_properties():
    h, g = WO.H, WO.G
    assert abs(np.sum(h) - math.sqrt(2)) < 1e-15
    assert abs(h @ h - 1) < 1e-15 and abs(g @ g - 1) < 1e-15
    assert abs(h[:2] @ h[2:]) < 1e-15                       # shift by 2 orthogonal
    assert abs(h @ g) < 1e-15 and abs(h[2:] @ g[:2]) < 1e-15 and abs(h[:2] @ g[2:]) < 1e-15
    n = np.arange(4)
    assert abs(np.sum(g)) < 1e-15 and abs(np.sum(n * g)) < 1e-14  # two vanishing moments


@pytest.mark.parametrize("n,levels", [(8, 1), (8, 3), (16, 2), (16, 4)])
def test_dense_matrix_is_orthogonal_and_idwt_is_its_transpose(n, levels):
    W = WO.dense_matrix(n, levels)
    assert np.max(np.abs(W.T @ W - np.eye(n * n))) < 1e-12
    rng = np.random.default_rng(n + levels)
    c = rng.standard_normal((n, n))
    assert np.max(np.abs(WO.idwt2(c, levels).ravel() - W.T @ c.ravel())) < 1e-12
    u = rng.standard_normal((n, n))
    assert np.max(np.abs(WO.idwt2(WO.dwt2(u, levels), levels) - u)) < 1e-12


def test_ramp_details_vanish_and_constant_maps_to_ll():
    n = 32
    y, x = np.mgrid[0:n, 0:n].astype(float)
    c = WO.dwt2(0.3 * x + 0.1 * y, 1)
    h = n // 2
    # the 4-tap support wraps only for the last output index along each axis
    assert np.max(np.abs(c[:h - 1, h:n - 1])) < 1e-12      # HL (detail along x)
    assert np.max(np.abs(c[h:n - 1, :h - 1])) < 1e-12      # LH (detail along y)
    k = WO.dwt2(np.full((n, n), 1.7), 3)
    m = n >> 3
    assert np.allclose(k[:m, :m], 1.7 * 8) and np.max(np.abs(k[m:, :])) < 1e-12 and np.max(np.abs(k[:, m:])) < 1e-12


def test_separable_abs_sums_match_dense():
    from oracle.wavelet_oracle import abs_sums
    for n, levels in [(16, 1), (16, 3), (32, 4)]:
        rows, cols = abs_sums(n, levels)
        r2, c2 = separable_abs_sums(n, levels)
        assert np.max(np.abs(rows - r2)) < 1e-12 and np.max(np.abs(cols - c2)) < 1e-12


def separable_abs_sums(n, levels):
    """The formula of the CUDA path: 1-D level operators built densely, then tensor
    products.  Row sum of a coefficient = (sum |a|)(sum |b|) of its two 1-D rows; column
    sum at pixel (y, x) = sum over subbands of colsum_y(y) * colsum_x(x)."""
    def analysis(M):
        A = np.zeros((M, M))
        for k in range(M // 2):
            for t in range(4):
                A[k, (2 * k + t) % M] += WO.H[t]
                A[M // 2 + k, (2 * k + t) % M] += WO.G[t]
        return A
    low = np.eye(n)
    ops = []                  # per level: (low rows, high rows), each (M/2 x n)
    M = n
    for _ in range(levels):
        A = analysis(M)
        lo, hi = A[:M // 2] @ low, A[M // 2:] @ low
        ops.append((lo, hi))
        low = lo
        M //= 2
    rows = np.zeros((n, n))
    cols = np.zeros((n, n))
    M = n
    for l, (lo, hi) in enumerate(ops):
        h2 = M // 2
        rl, rh = np.abs(lo).sum(1), np.abs(hi).sum(1)
        cl, ch = np.abs(lo).sum(0), np.abs(hi).sum(0)
        last = l == levels - 1
        # blocks of the Mallat layout: [y-rows, x-cols]
        rows[:h2, h2:M] = np.outer(rl, rh)       # HL: low y, high x
        rows[h2:M, :h2] = np.outer(rh, rl)       # LH
        rows[h2:M, h2:M] = np.outer(rh, rh)      # HH
        cols += np.outer(cl, ch) + np.outer(ch, cl) + np.outer(ch, ch)
        if last:
            rows[:h2, :h2] = np.outer(rl, rl)
            cols += np.outer(cl, cl)
        M = h2
    return rows, cols


def test_wavelet_pdhg_converges_and_alpha_limit():
    rng = np.random.default_rng(3)
    n, levels = 8, 2
    f = rng.uniform(0, 1, n * n)
    Kf = lambda u: np.asarray(u).ravel()
    KTf = lambda q: np.asarray(q).reshape(n, n)
    kcol = np.ones(n * n)
    krow = np.ones(n * n)
    sq, sr, tu = WO.wavelet_steps(kcol, krow, n, levels)
    u, q, r, hist = WO.pdhg_wavelet(Kf, KTf, f, n, levels, 0.05, 3000, sq, sr, tu, gap_every=100)
    assert hist[-1][2] < 1e-8
    # with K = I the solution is soft-thresholding in the orthonormal basis (closed form)
    c = WO.dwt2(f.reshape(n, n), levels)
    ref = WO.idwt2(np.sign(c) * np.maximum(np.abs(c) - 0.05, 0.0), levels)
    assert np.max(np.abs(u - ref)) < 1e-6
