"""Pins for the FP64 oracle of the learned warm start (oracle/unet_oracle.py), each
against something other than the oracle's own formulas:

* conv3x3 against scipy.signal.correlate2d (a library routine), channel by channel;
* conv3x3_backward, unet_backward and mse_loss against central finite differences of
  the forward maps;
* avgpool2 / upsample2 against hand-written arrays, and their adjoints by the identity
  <A x, y> = <x, A^T y>;
* bf16_round against hand-computed ties and against torch's bfloat16 conversion;
* adam_step against its closed-form first step and by minimising a quadratic;
* the warm-start maps: features of data from a constant image give that constant
  (the diagonal scalings of K reduce to 1 where the sums are positive); the state's q is a
  fixed point of the data prox of Sec. 3.2; target inverts state inside the balls.
"""
import math

import numpy as np
import pytest
import scipy.signal

import oracle as O
from oracle import unet_oracle as U


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3x3_matches_correlate2d():
    rng = _rng(1)
    x = rng.standard_normal((2, 7, 5, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for n in range(2):
        for o in range(4):
            acc = np.full((7, 5), b[o])
            for c in range(3):
                acc += scipy.signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same", boundary="fill")
            ref[n, :, :, o] = acc
    assert np.max(np.abs(y - ref)) < 1e-12
    assert np.max(np.abs(U.conv3x3(x, w, b, relu=True) - np.maximum(ref, 0.0))) < 1e-12


def test_conv3x3_backward_matches_finite_differences():
    rng = _rng(2)
    x = rng.standard_normal((2, 5, 6, 3))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    dz = rng.standard_normal((2, 5, 6, 2))

    def L(x_, w_, b_):
        return float(np.sum(dz * U.conv3x3(x_, w_, b_)))

    dx, dw, db = U.conv3x3_backward(x, w, dz)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 4, 5, 2), (0, 2, 3, 1), (1, 0, 5, 0)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert abs((L(x + e, w, b) - L(x - e, w, b)) / (2 * h) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 2, 2), (0, 1, 2, 1), (1, 0, 1, 0)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert abs((L(x, w + e, b) - L(x, w - e, b)) / (2 * h) - dw[idx]) < 1e-6
    for o in range(2):
        e = np.zeros_like(b)
        e[o] = h
        assert abs((L(x, w, b + e) - L(x, w, b - e)) / (2 * h) - db[o]) < 1e-6


def test_pool_and_upsample_hand_values_and_adjoints():
    x = np.arange(16, dtype=np.float64).reshape(1, 4, 4, 1)
    assert np.array_equal(U.avgpool2(x)[0, :, :, 0], np.array([[2.5, 4.5], [10.5, 12.5]]))
    s = np.array([[1.0, 2.0], [3.0, 4.0]]).reshape(1, 2, 2, 1)
    assert np.array_equal(U.upsample2(s)[0, :, :, 0],
                          np.array([[1, 1, 2, 2], [1, 1, 2, 2], [3, 3, 4, 4], [3, 3, 4, 4]], dtype=float))
    rng = _rng(3)
    a = rng.standard_normal((2, 6, 4, 3))
    c = rng.standard_normal((2, 3, 2, 3))
    assert abs(np.sum(U.avgpool2(a) * c) - np.sum(a * U.avgpool2_adjoint(c))) < 1e-12
    assert abs(np.sum(U.upsample2(c) * a) - np.sum(c * U.upsample2_adjoint(a))) < 1e-12


def test_bf16_round_ties_and_library():
    one = 1.0
    assert U.bf16_round(one) == 1.0
    assert U.bf16_round(1.0 + 2.0 ** -8) == 1.0                  # tie -> even (down)
    assert U.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # tie -> even (up)
    assert U.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert U.bf16_round(-3.0) == -3.0
    torch = pytest.importorskip("torch")
    v = _rng(4).standard_normal(10000) * 10.0 ** _rng(5).integers(-20, 20, 10000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(v), ref)


def _tiny(seed=6, levels=3, base=2, cin=2, cout=3):
    rng = _rng(seed)
    n = sum(c * 9 * i + c for _, c, i in U.unet_layout(cin, cout, base, levels))
    flat = rng.standard_normal(n) * 0.5
    x = rng.standard_normal((2, 8, 8, cin))
    t = rng.standard_normal((2, 8, 8, cout))
    wc = np.array([1.0, 2.0, 0.5])[:cout]
    return flat, x, t, wc


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_unet_backward_matches_finite_differences(levels):
    flat, x, t, wc = _tiny(levels=levels)
    cin, cout, base = 2, 3, 2

    def loss(v):
        y, _ = U.unet_forward(x, U.params_unflatten(v, cin, cout, base, levels), levels)
        return U.mse_loss(y, t, wc)[0]

    y, cache = U.unet_forward(x, U.params_unflatten(flat, cin, cout, base, levels), levels)
    _, dy = U.mse_loss(y, t, wc)
    g = U.params_flatten(U.unet_backward(dy, cache, levels), cin, cout, base, levels)
    rng = _rng(7)
    h = 1e-6
    for i in rng.choice(flat.size, 30, replace=False):
        e = np.zeros_like(flat)
        e[i] = h
        fd = (loss(flat + e) - loss(flat - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd)


def test_mse_gradient_matches_finite_differences():
    rng = _rng(8)
    y = rng.standard_normal((1, 3, 2, 3))
    t = rng.standard_normal((1, 3, 2, 3))
    wc = np.array([0.5, 1.0, 3.0])
    _, d = U.mse_loss(y, t, wc)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 2, 1, 2), (0, 1, 0, 1)]:
        e = np.zeros_like(y)
        e[idx] = h
        fd = (U.mse_loss(y + e, t, wc)[0] - U.mse_loss(y - e, t, wc)[0]) / (2 * h)
        assert abs(fd - d[idx]) < 1e-8


def test_adam_first_step_closed_form_and_quadratic():
    g = np.array([3.0, -0.2, 1e-3, 0.0])
    w1, m, v = U.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), t=1, lr=0.01)
    # bias-corrected first step: lr g / (|g| + eps)
    assert np.allclose(w1, -0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # minimises 1/2 (w - 3)^2
    w, m, v = np.array([0.0]), np.zeros(1), np.zeros(1)
    for t in range(1, 3001):
        w, m, v = U.adam_step(w, w - 3.0, m, v, t, lr=0.01)
    assert abs(w[0] - 3.0) < 1e-3


def _geom(n=8, n_det=6, n_t=12, m=32):
    ang = 2 * math.pi * (np.arange(n_det) + 0.5) / n_det
    det = np.stack([1.2 * np.cos(ang), 1.2 * np.sin(ang)], 1)
    return O.Geometry(n=n, det_xy=det, n_t=n_t, r0=0.0, dr=(1.2 + math.sqrt(2)) / n_t, quad_m=m)


def test_warm_features_of_constant_image():
    g = _geom()
    f = O.forward(g, np.full((8, 8), 0.7))
    x = U.warm_features(g, f)
    kcol = O.adjoint(g, np.ones((g.n_det, g.n_t)))
    inside = kcol > 0
    assert np.all(inside)
    assert np.max(np.abs(x[..., 0][inside] - 0.7)) < 1e-12
    assert abs(x[..., 1].max() - 1.0) < 1e-15 and x[..., 1].min() > 0
    assert not np.any(x[..., 2:])


@pytest.mark.parametrize("reg", [0, 1])
def test_warm_state_is_a_data_prox_fixed_point_and_target_inverts_it(reg):
    g = _geom()
    rng = _rng(9)
    n, S = g.n, g.n_det * g.n_t
    f = rng.standard_normal(S)
    alpha, beta = 0.05, 0.5
    pred = rng.standard_normal((n, n, 8)) * 0.3   # inside the unit balls mostly
    x, y = U.warm_state(g, pred, reg, alpha, beta, f)
    q = y[:S]
    Ku = O.forward(g, x[:n * n].reshape(n, n)).ravel()
    for sig in (0.1, 1.0, 7.0):
        assert np.max(np.abs(O.prox_f1_conj(q + sig * Ku, sig, f) - q)) < 1e-12
    # projections keep every dual vector inside its ball
    r = y[S:S + 2 * n * n].reshape(2, -1)
    assert np.all(np.hypot(r[0], r[1]) <= alpha * (1 + 1e-12))
    t = U.warm_target(n, S, x, y, reg, alpha, beta)
    small = np.hypot(pred[..., 3], pred[..., 4]) < 1.0
    assert np.allclose(t[..., 0], pred[..., 0], atol=1e-15)
    assert np.allclose(t[..., 3][small], pred[..., 3][small], atol=1e-12)
    if reg == 1:
        assert np.allclose(t[..., 1:3], pred[..., 1:3], atol=1e-12)
        small3 = np.sqrt(np.sum(pred[..., 5:8] ** 2, axis=-1)) < 1.0
        assert np.allclose(t[..., 5:8][small3], pred[..., 5:8][small3], atol=1e-12)
