"""Parity of the learned warm start's CUDA path (include/pat_unet.h) with the FP64 oracle.

Inputs are rounded to bfloat16 once and both sides read those values.  The oracle then
computes in FP64, and the GPU accumulates in FP32 on the tensor cores.  Tolerances:
- Single convolutions and their gradients are held element by element to
  2e-5 * sum|terms|.  The FP32 accumulation of up to 9 * 136 products stays well inside
  that.
- The whole network is compared with the oracle's bfloat16 emulation (the same rounding
  points).  Its tolerance is a relative L2 error of 1e-2 on the output and 3e-2 on the
  gradients, because one bf16 ulp (2^-8) of a stored activation propagates.
- Adam's first step is lr * g / (|g| + eps), so every weight with a clearly non-zero
  gradient moves by lr against its sign.
- The warm-start maps match the oracle to the FP32 error of K and to one bf16 ulp of
  the features.
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import pat_oracle as O
from oracle import unet_oracle as U

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1707_02245_gb300 as P  # noqa: E402
from paper_1707_02245_gb300 import warmstart as WS  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1707_02245_gb300 import build
    build.build()
    P.load()


def bf16(a):
    """(device bf16 tensor, the same values as float64 on the host)."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(torch.bfloat16).to(DEV)
    return t, t.float().cpu().numpy().astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().float().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CONV_CASES = [
    # B, H, W, cin, cout, relu
    (2, 13, 17, 8, 8, False),
    (2, 13, 17, 24, 40, True),
    (3, 40, 36, 96, 136, True),
    (1, 1, 1, 8, 8, False),
    (2, 5, 130, 16, 64, True),
    (1, 9, 7, 384, 128, False),
    # shapes that take the tensor-memory kernels: every N tile width (32, 64, 128, 256 for
    # the weight gradient), several tiles along x (W > 128) and ragged tiles
    (2, 16, 20, 64, 32, True),
    (1, 12, 10, 32, 64, False),
    (1, 12, 10, 64, 256, True),
    (1, 3, 200, 64, 64, False),
    (2, 13, 17, 64, 64, True),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_forward_matches_oracle(case):
    B, H, W, ci, co, relu = case
    rng = np.random.default_rng(hash(case) % 2**32)
    xt, x = bf16(rng.standard_normal((B, H, W, ci)))
    wt, w = bf16(rng.standard_normal((co, 3, 3, ci)) * 0.2)
    b = rng.standard_normal(co)
    y = torch.empty(B, H, W, co, device=DEV)
    P.pat_conv3x3_forward(xt, B, H, W, ci, wt, dev(b), co, relu, y)
    ref = U.conv3x3(x, w, b.astype(np.float32).astype(np.float64), relu=relu)
    bound = U.conv3x3(np.abs(x), np.abs(w), np.abs(b)) * 2e-5 + 1e-6
    err = np.abs(host(y) - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("case", [(2, 256, 256, 64, 64, True), (8, 64, 64, 128, 256, False)])
def test_conv_forward_many_tiles_per_cta_matches_oracle(case):
    """Shapes of the benchmark's network, where each persistent CTA of the tensor-memory
    kernel takes several tiles (1 024 and 256 x 2 tiles over 152 CTAs), so its stage ring
    and its four TMEM accumulators wrap around; every output is checked."""
    B, H, W, ci, co, relu = case
    rng = np.random.default_rng(7 + ci)
    xt, x = bf16(rng.standard_normal((B, H, W, ci)))
    wt, w = bf16(rng.standard_normal((co, 3, 3, ci)) * 0.1)
    b = rng.standard_normal(co)
    y = torch.empty(B, H, W, co, device=DEV)
    P.pat_conv3x3_forward(xt, B, H, W, ci, wt, dev(b), co, relu, y)
    ref = U.conv3x3(x, w, b.astype(np.float32).astype(np.float64), relu=relu)
    bound = U.conv3x3(np.abs(x), np.abs(w), np.abs(b)) * 2e-5 + 1e-6
    err = np.abs(host(y) - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_backward_data_matches_oracle(case):
    B, H, W, ci, co, _ = case
    rng = np.random.default_rng(hash(case) % 2**32 + 1)
    dyt, dy = bf16(rng.standard_normal((B, H, W, co)))
    wt, w = bf16(rng.standard_normal((co, 3, 3, ci)) * 0.2)
    dx = torch.empty(B, H, W, ci, device=DEV)
    P.pat_conv3x3_backward_data(dyt, B, H, W, co, wt, ci, dx)
    ref, _, _ = U.conv3x3_backward(np.zeros((B, H, W, ci)), w, dy)
    bound, _, _ = U.conv3x3_backward(np.zeros((B, H, W, ci)), np.abs(w), np.abs(dy))
    err = np.abs(host(dx) - ref)
    assert np.all(err <= 2e-5 * bound + 1e-6), float(np.max(err / (2e-5 * bound + 1e-6)))


@pytest.mark.parametrize("case", CONV_CASES + [(4, 64, 64, 32, 32, False)])
def test_conv_backward_weight_matches_oracle(case):
    B, H, W, ci, co, _ = case
    rng = np.random.default_rng(hash(case) % 2**32 + 2)
    xt, x = bf16(rng.standard_normal((B, H, W, ci)))
    dyt, dy = bf16(rng.standard_normal((B, H, W, co)))
    dw = torch.empty(co, 3, 3, ci, device=DEV)
    db = torch.empty(co, device=DEV)
    P.pat_conv3x3_backward_weight(xt, dyt, B, H, W, ci, co, dw, db)
    _, rw, rb = U.conv3x3_backward(x, np.zeros((co, 3, 3, ci)), dy)
    _, bw, bb = U.conv3x3_backward(np.abs(x), np.zeros((co, 3, 3, ci)), np.abs(dy))
    ew = np.abs(host(dw) - rw)
    eb = np.abs(host(db) - rb)
    assert np.all(ew <= 2e-5 * bw + 1e-6), float(np.max(ew / (2e-5 * bw + 1e-6)))
    assert np.all(eb <= 2e-5 * bb + 1e-6)


NET = dict(in_ch=8, out_ch=8, base_ch=8, levels=3)


def _net_and_inputs(seed, B=2, H=16, W=24, **over):
    cfg = dict(NET, **over)
    net = WS.UNet(base_ch=cfg["base_ch"], levels=cfg["levels"], seed=seed, in_ch=cfg["in_ch"], out_ch=cfg["out_ch"])
    rng = np.random.default_rng(seed)
    xt, x = bf16(rng.standard_normal((B, H, W, cfg["in_ch"])))
    return net, cfg, xt, x


def _oracle_params(net, cfg):
    return U.params_unflatten(net.get_params().astype(np.float64), cfg["in_ch"], cfg["out_ch"], cfg["base_ch"],
                              cfg["levels"])


@pytest.mark.parametrize("levels", [1, 3, 4])
def test_unet_forward_backward_match_oracle(levels):
    B, H, W = 2, 16, 24
    net, cfg, xt, x = _net_and_inputs(11 + levels, B, H, W, levels=levels)
    y = torch.empty(B, H, W, cfg["out_ch"], device=DEV)
    net.forward(xt, B, H, W, y)
    prm = _oracle_params(net, cfg)
    ref, cache = U.unet_forward(x, prm, levels, bf16=True)
    assert rel_l2(host(y), ref) < 1e-2
    dy = np.random.default_rng(5).standard_normal(ref.shape)
    g = torch.empty(net.num_params, device=DEV)
    P.pat_unet_backward(net.handle, dev(dy), g)
    rg = U.params_flatten(U.unet_backward(dy.astype(np.float32).astype(np.float64), cache, levels, bf16=True),
                          cfg["in_ch"], cfg["out_ch"], cfg["base_ch"], levels)
    gg = host(g)
    assert rel_l2(gg, rg) < 3e-2
    # every conv's weight gradient separately
    k = 0
    for name, co, ci in U.unet_layout(cfg["in_ch"], cfg["out_ch"], cfg["base_ch"], levels):
        nw = co * 9 * ci
        assert rel_l2(gg[k:k + nw], rg[k:k + nw]) < 5e-2, name
        k += nw + co
    net.close()


def test_benchmark_width_unet_matches_oracle_within_rounding_noise():
    """The benchmark's network (C0 = 32, 4 levels: channels up to 384, the wide layers on
    the tensor-memory kernels) against the oracle's bf16 emulation.  Rounding a stored
    activation to bf16 turns an FP32-level difference in a convolution sum into a jump of
    one bf16 ulp, and such flips propagate: perturbing every convolution output of the
    oracle itself by a relative 3e-6 (the order of FP32 accumulation error over 9 x 384
    terms) moves its output by 3-5e-3 and its gradients by 5-11e-2 at C0 = 8, 16 and 32.
    The bounds below sit above that noise; a wiring error gives differences of order 1."""
    B, H, W = 2, 16, 24
    net, cfg, xt, x = _net_and_inputs(15, B, H, W, levels=4, base_ch=32)
    y = torch.empty(B, H, W, cfg["out_ch"], device=DEV)
    net.forward(xt, B, H, W, y)
    prm = _oracle_params(net, cfg)
    ref, cache = U.unet_forward(x, prm, 4, bf16=True)
    assert rel_l2(host(y), ref) < 1e-2
    dy = np.random.default_rng(5).standard_normal(ref.shape)
    g = torch.empty(net.num_params, device=DEV)
    P.pat_unet_backward(net.handle, dev(dy), g)
    rg = U.params_flatten(U.unet_backward(dy.astype(np.float32).astype(np.float64), cache, 4, bf16=True),
                          cfg["in_ch"], cfg["out_ch"], cfg["base_ch"], 4)
    assert rel_l2(host(g), rg) < 0.15
    net.close()


def test_adam_first_step_and_training_reduces_loss():
    B, H, W = 2, 16, 16
    net, cfg, xt, x = _net_and_inputs(21, B, H, W)
    p0 = net.get_params().astype(np.float64)
    rng = np.random.default_rng(22)
    t = rng.standard_normal((B, H, W, cfg["out_ch"])) * 0.5
    cw = np.linspace(0.5, 2.0, cfg["out_ch"])
    # oracle gradient at the initial parameters
    prm = _oracle_params(net, cfg)
    y, cache = U.unet_forward(x, prm, cfg["levels"], bf16=True)
    loss0, dy = U.mse_loss(y, t, cw)
    rg = U.params_flatten(U.unet_backward(dy, cache, cfg["levels"], bf16=True), cfg["in_ch"], cfg["out_ch"],
                          cfg["base_ch"], cfg["levels"])
    lr = 1e-3
    loss = torch.zeros(1, device=DEV)
    tt = dev(t)
    P.pat_unet_train_step(net.handle, xt, tt, cw.astype(np.float32), B, H, W, lr, loss)
    assert abs(float(loss.item()) - loss0) < 1e-2 * loss0
    d = net.get_params().astype(np.float64) - p0
    clear = np.abs(rg) > 5e-2 * np.abs(rg).max()
    assert clear.sum() > 50
    assert np.all(np.abs(np.abs(d[clear]) - lr) < 1e-3 * lr + 1e-9)
    assert np.all(np.sign(d[clear]) == -np.sign(rg[clear]))
    first = float(loss.item())
    for _ in range(60):
        P.pat_unet_train_step(net.handle, xt, tt, cw.astype(np.float32), B, H, W, 3e-3, loss)
    assert float(loss.item()) < 0.5 * first
    net.close()


def test_set_params_round_trip_and_forward_determinism():
    B, H, W = 1, 8, 8
    net, cfg, xt, x = _net_and_inputs(31, B, H, W)
    p = net.get_params()
    net.set_params(p * 0.5)
    assert np.array_equal(net.get_params(), (p * 0.5).astype(np.float32))
    y1 = torch.empty(B, H, W, cfg["out_ch"], device=DEV)
    y2 = torch.empty_like(y1)
    net.forward(xt, B, H, W, y1)
    net.forward(xt, B, H, W, y2)
    assert torch.equal(y1, y2)
    with pytest.raises(P.PatError):
        net.forward(xt, B, 6, 8, y1)   # 6 is not a multiple of 2^(levels-1) = 4
    net.close()


def _small_geometry(n=16, n_det=12, n_t=24, m=64):
    det = S.detectors_full_circle(n_det, 1.2)
    r0, dr = S.radial_sampling(det, n_t)
    og = O.Geometry(n=n, det_xy=det, n_t=n_t, r0=r0, dr=dr, quad_m=m)
    return og, P.Geometry(n, det, n_t, r0, dr, m)


def test_warm_start_features_match_oracle():
    og, g = _small_geometry()
    rng = np.random.default_rng(41)
    f = rng.standard_normal(og.n_det * og.n_t).astype(np.float32)
    x = torch.empty(og.n, og.n, 8, dtype=torch.bfloat16, device=DEV)
    P.pat_warm_start_features(g.handle, dev(f), x, 8)
    ref = U.warm_features(og, f.astype(np.float64))
    got = host(x)
    tol = 2.0 ** -7 * np.abs(ref) + 1e-6   # one bf16 ulp of FP32-close values
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))
    g.close()


@pytest.mark.parametrize("reg", [P.PAT_TV, P.PAT_TGV])
def test_warm_start_state_and_target_match_oracle(reg):
    og, g = _small_geometry()
    n, S_ = og.n, og.n_det * og.n_t
    rng = np.random.default_rng(43 + reg)
    pred = (rng.standard_normal((n, n, 8)) * 0.6).astype(np.float32)
    f = rng.standard_normal(S_).astype(np.float32)
    alpha, beta = 0.05, 0.5
    prm = P.make_params(reg=reg, alpha=alpha, beta=beta)
    nx = n * n * (3 if reg == P.PAT_TGV else 1)
    ny = S_ + n * n * (5 if reg == P.PAT_TGV else 2)
    x0 = torch.empty(nx, device=DEV)
    y0 = torch.empty(ny, device=DEV)
    P.pat_warm_start_state(g.handle, dev(pred), 8, prm, dev(f), x0, y0)
    rx, ry = U.warm_state(og, pred.astype(np.float64), reg, alpha, beta, f.astype(np.float64))
    hx, hy = host(x0), host(y0)
    assert np.max(np.abs(hx - rx)) < 1e-6
    assert rel_l2(hy[:S_], ry[:S_]) < 1e-4                 # q = K u - f
    assert np.max(np.abs(hy[S_:] - ry[S_:])) < 1e-6 * (1 + np.abs(ry[S_:]).max())
    t = torch.empty(n, n, 8, device=DEV)
    P.pat_warm_start_target(g.handle, x0, y0, prm, t, 8)
    rt = U.warm_target(n, S_, hx, hy, reg, alpha, beta)
    assert np.max(np.abs(host(t) - rt)) < 1e-5 * (1 + np.abs(rt).max())
    g.close()


def test_warm_start_one_call_equals_its_steps():
    og, g = _small_geometry()
    n, S_ = og.n, og.n_det * og.n_t
    net = WS.UNet(base_ch=8, levels=3, seed=51)
    f = dev(np.random.default_rng(52).standard_normal(S_))
    prm = P.make_params(reg=P.PAT_TGV, alpha=0.02, beta=0.04)
    x0a, y0a = torch.empty(3 * n * n, device=DEV), torch.empty(S_ + 5 * n * n, device=DEV)
    P.pat_warm_start(g.handle, net.handle, f, prm, x0a, y0a)
    feats = torch.empty(n, n, 8, dtype=torch.bfloat16, device=DEV)
    P.pat_warm_start_features(g.handle, f, feats, 8)
    pred = torch.empty(n, n, 8, device=DEV)
    net.forward(feats, 1, n, n, pred)
    x0b, y0b = torch.empty_like(x0a), torch.empty_like(y0a)
    P.pat_warm_start_state(g.handle, pred, 8, prm, f, x0b, y0b)
    torch.cuda.synchronize()
    assert torch.equal(x0a, x0b) and torch.equal(y0a, y0b)
    net.close()
    g.close()


def test_zz_no_tensor_memory_wait_ran_out():
    """Every bounded mbarrier wait of the tensor-memory convolutions in this module's runs
    completed (a wait that ran out would have ended its CTA without output)."""
    assert P.pat_nn_wait_timeouts() == 0
