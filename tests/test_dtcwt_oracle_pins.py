"""Pins of the DT-CWT oracle (oracle/dtcwt_oracle.py) against facts that do not come from
its own formulas: the filters' closed-form properties, the already-pinned Daubechies DWT
of the wavelet oracle, circular shifts, orthogonality and the tight-frame property by
dense matrices, the directional selectivity that defines the dual tree (Sec. 2.2), the
Moreau identity of the dual prox, and an independent dual solver for K = I."""
import math

import numpy as np
import pytest

from oracle import dtcwt_oracle as D
from oracle import wavelet_oracle as WO


def test_qshift_filter_closed_form():
    h = D.QSHIFT4
    assert h.sum() == pytest.approx(math.sqrt(2.0), abs=1e-15)
    assert (h * h).sum() == pytest.approx(1.0, abs=1e-15)
    assert h[0] * h[2] + h[1] * h[3] == pytest.approx(0.0, abs=1e-15)     # even shifts orthogonal
    assert sum((-1) ** n * h[n] for n in range(4)) == pytest.approx(0.0, abs=1e-15)   # zero at pi
    # centre a quarter sample before the midpoint 1.5: the Q-shift property
    assert (np.arange(4) * h).sum() / h.sum() == pytest.approx(1.25, abs=1e-15)
    # tree b's filter (reversed) has its centre a quarter sample after: half a sample apart
    hb = h[::-1]
    assert (np.arange(4) * hb).sum() / hb.sum() - 1.25 == pytest.approx(0.5, abs=1e-15)


def test_level_one_filter_is_the_pinned_daubechies_filter():
    assert np.allclose(D.D4, WO.H, atol=1e-16, rtol=0)
    assert np.allclose(D.highpass(D.D4), WO.G, atol=1e-16, rtol=0)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_tree_aa_with_daubechies_filters_is_the_dwt(levels):
    # with the Daubechies filter at every level, tree aa is the wavelet oracle's DWT
    u = np.random.default_rng(1).standard_normal((16, 16))
    T = D.tree_transform(u, levels, 0, (D.D4, D.D4))
    assert np.abs(T - WO.dwt2(u, levels)).max() < 1e-13


def test_tree_b_level_one_is_the_dwt_of_the_shifted_image():
    # tree b's level-1 filters are tree a's delayed by one sample
    u = np.random.default_rng(2).standard_normal((16, 16))
    for t, shift in ((1, (-1, 0)), (2, (0, -1)), (3, (-1, -1))):
        T = D.tree_transform(u, 1, t, (D.D4, D.D4))
        assert np.abs(T - WO.dwt2(np.roll(u, shift, axis=(0, 1)), 1)).max() < 1e-13, t


@pytest.mark.parametrize("n,levels", [(8, 1), (8, 3), (16, 2)])
def test_every_tree_is_orthonormal(n, levels):
    for t in range(4):
        M = np.stack([D.tree_transform(e.reshape(n, n), levels, t).ravel() for e in np.eye(n * n)], axis=1)
        assert np.abs(M.T @ M - np.eye(n * n)).max() < 1e-12, t
        c = np.random.default_rng(t).standard_normal((n, n))
        assert np.abs(D.tree_transpose(c, levels, t) - (M.T @ c.ravel()).reshape(n, n)).max() < 1e-12


@pytest.mark.parametrize("n,levels", [(8, 2), (16, 3)])
def test_tight_frame_by_dense_matrix(n, levels):
    W = D.dense_matrix(n, levels)
    assert W.shape == (4 * n * n, n * n)
    assert np.abs(W.T @ W - np.eye(n * n)).max() < 1e-12          # W^T W = I, ||W|| = 1
    assert np.linalg.norm(W, 2) == pytest.approx(1.0, abs=1e-12)
    c = np.random.default_rng(3).standard_normal((4, n, n))
    assert np.abs(D.idtcwt2(c, levels) - (W.T @ c.ravel()).reshape(n, n)).max() < 1e-12


def test_perfect_reconstruction_and_parseval_at_size():
    u = np.random.default_rng(4).standard_normal((64, 64))
    C = D.dtcwt2(u, 4)
    assert np.abs(D.idtcwt2(C, 4) - u).max() < 1e-12
    assert np.linalg.norm(C) == pytest.approx(np.linalg.norm(u), rel=1e-13)


def test_combination_is_orthogonal():
    T = np.random.default_rng(5).standard_normal((4, 6, 6))
    C = D.combine(T)
    assert np.abs(D.uncombine(C) - T).max() < 1e-15
    assert np.linalg.norm(C) == pytest.approx(np.linalg.norm(T), rel=1e-15)


@pytest.mark.parametrize("level,ratio", [(2, 10.0), (3, 5.0)])
def test_directional_selectivity_separates_plus_and_minus_45_degrees(level, ratio):
    """The reason for the dual tree (Sec. 2.2): a cosine oriented at +45 degrees puts its
    diagonal energy into one complex subband and one at -45 degrees into the other, which
    a real separable DWT cannot do (its HH subband answers both alike)."""
    n, J = 64, 4
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    w = 2 * math.pi / 2 ** level * 0.75
    M = n >> (level - 1)
    hh = (slice(M // 2, M), slice(M // 2, M))
    e = {}
    for name, img in (("+", np.cos(w * (x + y) / math.sqrt(2))), ("-", np.cos(w * (x - y) / math.sqrt(2)))):
        C = D.dtcwt2(img, J)
        e[name] = ((C[0][hh] ** 2 + C[1][hh] ** 2).sum(), (C[2][hh] ** 2 + C[3][hh] ** 2).sum())
        dw = WO.dwt2(img, J)
        e[name + "dwt"] = (dw[hh] ** 2).sum()
    assert e["+"][0] > ratio * e["+"][1]
    assert e["-"][1] > ratio * e["-"][0]
    # the real DWT cannot tell them apart: its HH energies for the two orientations stay
    # within a factor 1.5 of each other
    assert max(e["+dwt"], e["-dwt"]) < 1.5 * min(e["+dwt"], e["-dwt"])


def test_l1_and_projection():
    rng = np.random.default_rng(6)
    n, J, alpha = 8, 2, 0.7
    C = rng.standard_normal((4, n, n))
    m = D.ll_mask(n, J)
    # ||.||_1 by a plain loop
    tot = 0.0
    for y in range(n):
        for x in range(n):
            if m[y, x]:
                tot += sum(abs(C[c, y, x]) for c in range(4))
            else:
                tot += math.hypot(C[0, y, x], C[1, y, x]) + math.hypot(C[2, y, x], C[3, y, x])
    assert D.l1(C, J) == pytest.approx(tot, rel=1e-14)
    # Moreau: C = prox_{alpha l1}(C) + P_alpha(C); the prox shrinks moduli by alpha
    P = D.project(C, alpha, J)
    S = C - P
    for y in range(n):
        for x in range(n):
            if m[y, x]:
                for c in range(4):
                    v = C[c, y, x]
                    assert S[c, y, x] == pytest.approx(np.sign(v) * max(abs(v) - alpha, 0.0), abs=1e-14)
            else:
                for a, b in ((0, 1), (2, 3)):
                    mod = math.hypot(C[a, y, x], C[b, y, x])
                    k = max(mod - alpha, 0.0) / mod
                    assert S[a, y, x] == pytest.approx(k * C[a, y, x], abs=1e-14)
                    assert S[b, y, x] == pytest.approx(k * C[b, y, x], abs=1e-14)
    assert np.all(np.hypot(P[0], P[1])[~m] <= alpha + 1e-15)


def test_abs_sums_match_the_dense_matrix():
    n, J = 8, 2
    A = np.abs(D.dense_matrix(n, J))
    rows, cols = D.abs_sums(n, J)
    assert np.abs(rows.ravel() - A.sum(axis=1)).max() < 1e-13
    assert np.abs(cols.ravel() - A.sum(axis=0)).max() < 1e-13


def test_pdhg_with_identity_matches_a_dual_projected_gradient_solver():
    """K = I: min_u 1/2 |u - f|^2 + alpha ||W u||_1.  Its dual is min over the product of
    discs (and LL intervals) of 1/2 |f - W^T r|^2 with u = f - W^T r; since ||W|| = 1,
    projected gradient with step 1 (accelerated, FISTA) converges.  Written independently
    of the PDHG loop."""
    n, J, alpha = 16, 3, 0.15
    rng = np.random.default_rng(7)
    y, x = np.mgrid[0:n, 0:n]
    f = ((x - 7.5) ** 2 + (y - 7.5) ** 2 < 30).astype(float) + 0.1 * rng.standard_normal((n, n))
    r = np.zeros((4, n, n))
    z, tk = r.copy(), 1.0
    for _ in range(3000):
        grad = -D.dtcwt2(f - D.idtcwt2(z, J), J)
        r_new = D.project(z - grad, alpha, J)
        tk1 = (1 + math.sqrt(1 + 4 * tk * tk)) / 2
        z = r_new + (tk - 1) / tk1 * (r_new - r)
        r, tk = r_new, tk1
    u_ref = f - D.idtcwt2(r, J)
    ones = np.ones(n * n)
    sq, sr, tu = D.cwt_steps(ones, ones, n, J)
    u, q, rr, hist = D.pdhg_cwt(lambda v: np.asarray(v).ravel(), lambda v: np.asarray(v).reshape(n, n), f, n, J,
                                alpha, 3000, sq, sr, tu, gap_every=500)
    # (a wrong step rule, e.g. separate steps for the two rows of a complex coefficient,
    # converges to another point: 1e-2 away, relative gap stuck at 6e-4)
    assert np.abs(u - u_ref).max() < 3e-4
    assert hist[-1][2] < 1e-5
