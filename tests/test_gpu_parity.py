"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 1e-4 for single applications of K and K^T and for the step
arrays, 1e-3 on the image after a fixed number of PDHG iterations (FP32 iterates),
and FP32-level agreement for one iteration from a given state.
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import pat_oracle as O
from tests.problems import make, oracle_geometry, oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1707_02245_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1707_02245_gb300 import build
    build.build()
    P.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def geometry_pair(n, det, n_t, r0, dr, m, extent=(-1.0, 1.0, -1.0, 1.0)):
    og = O.Geometry(n=n, det_xy=det, n_t=n_t, r0=r0, dr=dr, quad_m=m, xmin=extent[0], xmax=extent[1],
                    ymin=extent[2], ymax=extent[3])
    return og, P.Geometry(n, det, n_t, r0, dr, m, extent)


GEOMS = {
    "full_circle": lambda: (24, S.detectors_full_circle(12, 1.2), 40, 0.0, 2.62 / 40, 64),
    "ragged_odd": lambda: (33, S.detectors_full_circle(7, 1.3), 45, 0.0, 2.8 / 45, 50),
    "limited_arc": lambda: (32, S.detectors_limited_arc(128, 32, 90.0, 5, 1.2), 70, 0.0, 2.7 / 70, 96),
    "one_det_one_t": lambda: (16, np.array([[1.2, 0.1]]), 1, 1.1, 0.3, 128),
    "centre_det": lambda: (20, np.array([[0.03, -0.05], [0.5, 0.4]]), 33, 0.0, 0.05, 200),
    "n2": lambda: (2, np.array([[0.0, 1.5], [0.2, -1.1]]), 9, 0.0, 0.35, 40),
    "far_outside": lambda: (12, np.array([[4.0, 4.0]]), 8, 0.0, 0.2, 32),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_forward_adjoint_parity(name):
    n, det, n_t, r0, dr, m = GEOMS[name]()
    og, pg = geometry_pair(n, det, n_t, r0, dr, m)
    rng = np.random.default_rng(len(name))
    u = rng.standard_normal((n, n)).astype(np.float32)
    y = rng.standard_normal((len(det), n_t)).astype(np.float32)
    y_d = torch.empty(len(det), n_t, device=DEV)
    u_d = torch.empty(n, n, device=DEV)
    P.pat_forward(pg.handle, dev(u), y_d)
    P.pat_adjoint(pg.handle, dev(y), u_d)
    yk = O.forward(og, u.astype(np.float64))
    uk = O.adjoint(og, y.astype(np.float64))
    yg, ug = host(y_d), host(u_d)
    if name == "far_outside":
        assert np.all(yg == 0) and np.all(ug == 0)
        return
    assert rel_l2(yg, yk) <= 1e-4
    assert rel_l2(ug, uk) <= 1e-4
    # FP32 adjoint identity
    lhs, rhs = float(np.sum(yg * y)), float(np.sum(u * ug))
    assert abs(lhs - rhs) <= 1e-5 * (np.linalg.norm(yg) * np.linalg.norm(y))


def test_forward_adjoint_non_square_extent():
    det = np.array([[2.0, 0.0], [0.0, 2.5], [-1.5, -1.0]])
    og, pg = geometry_pair(20, det, 50, 0.2, 0.08, 80, extent=(-1.5, 1.0, -0.5, 1.5))
    u = np.random.default_rng(0).standard_normal((20, 20)).astype(np.float32)
    y_d = torch.empty(3, 50, device=DEV)
    P.pat_forward(pg.handle, dev(u), y_d)
    assert rel_l2(host(y_d), O.forward(og, u.astype(np.float64))) <= 1e-4


def test_forward_adjoint_full_size_sampled():
    """The 256^2, 256 x 512, M = 256 geometry: sampled rows of K u one by one, and K^T y
    for data supported on a few detectors."""
    w = S.workload("tgv256")
    og = oracle_geometry(w)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    rng = np.random.default_rng(1)
    u = (w["phantom"] + 0.1 * rng.standard_normal(w["phantom"].shape)).astype(np.float32)
    y_d = torch.empty(og.n_det, og.n_t, device=DEV)
    P.pat_forward(pg.handle, dev(u), y_d)
    yg = host(y_d).ravel()
    rows = rng.choice(og.n_det * og.n_t, size=96, replace=False)
    yk = O.forward_rows(og, u.astype(np.float64), rows)
    assert rel_l2(yg[rows], yk) <= 1e-4
    y = np.zeros((og.n_det, og.n_t), dtype=np.float32)
    dets = rng.choice(og.n_det, size=6, replace=False)
    y[dets] = rng.standard_normal((6, og.n_t))
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    P.pat_adjoint(pg.handle, dev(y), u_d)
    assert rel_l2(host(u_d), O.adjoint(og, y.astype(np.float64))) <= 1e-4


@pytest.mark.parametrize("reg", [0, 1, 2])
def test_steps_parity(reg):
    w = make("small", seed=reg, reg=reg)
    pb = oracle_problem(w)
    st = O.diag_steps(pb)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    n = w["n"]
    xi_d = dev(w["xi"]) if reg == 2 else None
    prm = P.make_params(reg=reg, alpha=w["alpha"], gamma=w["gamma"], xi=xi_d)
    sq = torch.empty(pb.f.size, device=DEV)
    tu = torch.empty(n, n, device=DEV)
    sr = torch.empty(n, n, device=DEV)
    ss = torch.empty(n, n, device=DEV)
    tv = torch.empty(2, n, n, device=DEV)
    P.pat_steps(pg.handle, prm, sq, tu, sr, ss, tv)
    # sig_q and tau_u are reciprocals of K sums: the operator tolerance applies (rows
    # that barely touch the grid carry the FP32 point-position error)
    assert rel_l2(host(sq), st.sig_q) <= 1e-4
    assert rel_l2(host(tu), st.tau_u) <= 1e-4
    assert rel_l2(host(sr), st.sig_r) <= 1e-6
    if reg == 1:
        assert rel_l2(host(ss), st.sig_s) <= 1e-6
        assert rel_l2(host(tv), st.tau_v) <= 1e-6


def _random_state(w, reg, rng, scale=0.3):
    n, S_ = w["n"], w["f"].size
    u = rng.uniform(0, 1, (n, n))
    v = scale * rng.standard_normal((2, n, n))
    q = scale * rng.standard_normal(S_)
    r = O.proj_ball(rng.standard_normal((2, n, n)), w["alpha"])
    s = O.proj_ball(rng.standard_normal((3, n, n)), w["alpha"] * w["beta"])
    ub = u + 0.1 * rng.standard_normal((n, n))
    vb = v + 0.1 * rng.standard_normal((2, n, n))
    tgv = reg == 1
    x = np.concatenate([u.ravel()] + ([v.ravel()] if tgv else []))
    xb = np.concatenate([ub.ravel()] + ([vb.ravel()] if tgv else []))
    y = np.concatenate([q, r.ravel()] + ([s.ravel()] if tgv else []))
    return dict(u=u, v=v if tgv else None, q=q, r=r, s=s if tgv else None, ub=ub, vb=vb if tgv else None,
                x=x.astype(np.float32), xb=xb.astype(np.float32), y=y.astype(np.float32))


def _with_xi(w, reg):
    assert reg != 2 or "xi" in w
    return w


@pytest.mark.parametrize("reg", [0, 1, 2])
def test_gap_parity_random_state(reg):
    w = _with_xi(make("small", seed=4, reg=reg, beta=0.5), reg)
    pb = oracle_problem(w)
    st = _random_state(w, reg, np.random.default_rng(7))
    f32 = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)  # noqa: E731
    ref = O.duality_gap(pb, f32(st["u"]), f32(st["q"]), f32(st["r"]), f32(st["v"]), f32(st["s"]))
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    prm = P.make_params(reg=reg, alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"],
                        xi=dev(w["xi"]) if reg == 2 else None)
    got = P.pat_duality_gap(pg.handle, dev(w["f"]), prm, dev(st["x"]), dev(st["y"]))
    scale = abs(ref["primal"]) + abs(ref["dual"])
    for k in ("primal", "dual", "gap"):
        assert abs(got[k] - ref[k]) <= 2e-6 * scale, (k, got[k], ref[k])


@pytest.mark.parametrize("reg", [0, 1, 2])
def test_one_iteration_from_state(reg):
    """One PDHG iteration from a random state (Algorithm 1 / 2 steps a1-a4)."""
    w = _with_xi(make("small", seed=5, reg=reg, beta=0.5), reg)
    n, S_ = w["n"], w["f"].size
    pb = oracle_problem(w)
    st = _random_state(w, reg, np.random.default_rng(11))
    f32 = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)  # noqa: E731
    ref = O.pdhg(pb, 1, x0={"u": f32(st["u"]), "v": f32(st["v"])},
                 y0={"q": f32(st["q"]), "r": f32(st["r"]), "s": f32(st["s"])},
                 xbar0={"u": f32(st["ub"]), "v": f32(st["vb"])})
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    nx, ny = st["x"].size, st["y"].size
    xo, xbo, yo = (torch.empty(k, device=DEV) for k in (nx, nx, ny))
    u_d = torch.empty(n, n, device=DEV)
    prm = P.make_params(reg=reg, alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"],
                        xi=dev(w["xi"]) if reg == 2 else None, iters=1, gap_every=0,
                        x0=dev(st["x"]), xbar0=dev(st["xb"]), y0=dev(st["y"]), x_out=xo, xbar_out=xbo, y_out=yo)
    x0d, xb0d, y0d = prm.x0_dev, prm.xbar0_dev, prm.y0_dev  # keep buffers alive  # noqa: F841
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert info["iters_done"] == 1
    xg, xbg, yg = host(xo), host(xbo), host(yo)
    assert rel_l2(xg[:n * n], ref.u) <= 2e-6
    assert rel_l2(host(u_d), ref.u) <= 2e-6
    assert rel_l2(xbg[:n * n], ref.ubar) <= 2e-6
    assert rel_l2(yg[:S_], ref.q) <= 2e-6
    assert rel_l2(yg[S_:S_ + 2 * n * n], ref.r) <= 2e-6
    if reg == 1:
        assert rel_l2(xg[n * n:], ref.v) <= 2e-6
        assert rel_l2(xbg[n * n:], ref.vbar) <= 2e-6
        assert rel_l2(yg[S_ + 2 * n * n:], ref.s) <= 2e-6


@pytest.mark.parametrize("reg", [0, 1, 2])
def test_fixed_iterations_small(reg):
    w = _with_xi(make("small", seed=6, reg=reg, beta=0.5), reg)
    iters = 60
    pb = oracle_problem(w)
    ref = O.pdhg(pb, iters, gap_every=20)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    prm = P.make_params(reg=reg, alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"],
                        xi=dev(w["xi"]) if reg == 2 else None, iters=iters, gap_every=20)
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert info["iters_done"] == iters and info["status"] == P.PAT_STATUS_MAXITER
    assert rel_l2(host(u_d), ref.u) <= 1e-3
    assert abs(info["gap"] - ref.gap["gap"]) <= 1e-4 * ref.gap["primal"]
    assert abs(info["residual"] - ref.residual) <= 1e-2 * ref.residual + 1e-7


@pytest.mark.parametrize("reg,ratio", [(0, 0.3), (1, 4.0), (2, 0.5)])
def test_step_ratio_matches_oracle_balanced_steps(reg, ratio):
    """tau -> s tau, sigma -> sigma / s on every block (pat_params.step_ratio)."""
    w = _with_xi(make("small", seed=9, reg=reg, beta=0.5), reg)
    iters = 60
    pb = oracle_problem(w)
    ref = O.pdhg(pb, iters, steps=O.balanced_steps(O.diag_steps(pb), ratio), gap_every=20)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    prm = P.make_params(reg=reg, alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"],
                        xi=dev(w["xi"]) if reg == 2 else None, iters=iters, gap_every=20, step_ratio=ratio)
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert rel_l2(host(u_d), ref.u) <= 1e-3
    assert abs(info["gap"] - ref.gap["gap"]) <= 1e-4 * ref.gap["primal"]
    # the exported steps carry the balance too
    st = O.balanced_steps(O.diag_steps(pb), ratio)
    tau = torch.empty(w["n"], w["n"], device=DEV)
    sq = torch.empty(w["det_xy"].shape[0] * w["n_t"], device=DEV)
    P.pat_steps(pg.handle, prm, sig_q=sq, tau_u=tau)
    assert rel_l2(host(tau), st.tau_u) <= 1e-4
    assert rel_l2(host(sq), st.sig_q) <= 1e-4


@pytest.mark.parametrize("reg", [0, 1, 2])
def test_adaptive_balance_matches_oracle(reg):
    """PAT_ADAPT_BALANCE: the same residual-balancing decisions as the oracle (the final s
    agrees), hence the same iterates."""
    w = _with_xi(make("small", seed=10, reg=reg, beta=0.5, alpha=0.2), reg)
    iters = 300
    pb = oracle_problem(w)
    ref = O.pdhg(pb, iters, gap_every=10, adapt=True)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    prm = P.make_params(reg=reg, alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"],
                        xi=dev(w["xi"]) if reg == 2 else None, iters=iters, gap_every=10, adapt=P.PAT_ADAPT_BALANCE)
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert ref.step_ratio != 1.0
    # each adjustment is sqrt of a residual ratio (FP32 terms, FP64 sums on the GPU), so
    # equal decisions leave s equal to a few 1e-4
    assert abs(info["step_ratio"] - ref.step_ratio) <= 2e-3 * ref.step_ratio
    assert rel_l2(host(u_d), ref.u) <= 1e-3


def test_tune_step_ratio_picks_the_smallest_probe_gap():
    w = make("small", seed=11, reg=1, beta=0.5)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    f = dev(w["f"])
    prm = P.make_params(reg=1, alpha=w["alpha"], beta=w["beta"], iters=5, gap_every=1)
    cands = [0.3, 1.0, 3.0, 10.0]
    best, gaps = P.pat_tune_step_ratio(pg.handle, f, prm, cands, 40)
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    single = []
    for s_ in cands:
        p1 = P.make_params(reg=1, alpha=w["alpha"], beta=w["beta"], iters=40, gap_every=0, step_ratio=s_)
        single.append(P.pat_reconstruct(pg.handle, f, p1, u_d)["rel_gap"])
    assert gaps == single                       # the probes are the single runs, bitwise
    assert best == cands[int(np.argmin(single))]
    with pytest.raises(P.PatError):
        P.pat_tune_step_ratio(pg.handle, f, prm, [1.0, -2.0], 40)


def test_replays_end_once_every_problem_has_stopped():
    """A generous iteration cap costs nothing after convergence: the graph replays stop
    within two chunks of the last problem's stop, and the result is unchanged."""
    w = make("small", seed=12, reg=0)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    f = dev(w["f"])
    u_a = torch.empty(w["n"], w["n"], device=DEV)
    u_b = torch.empty_like(u_a)
    pa = P.make_params(reg=0, alpha=w["alpha"], iters=2000, tol=1e-2, gap_every=10)
    pb = P.make_params(reg=0, alpha=w["alpha"], iters=400000, tol=1e-2, gap_every=10)
    ia = P.pat_reconstruct(pg.handle, f, pa, u_a)
    l0 = P.pat_kernel_launches()
    ib = P.pat_reconstruct(pg.handle, f, pb, u_b)
    launches = P.pat_kernel_launches() - l0
    assert ia["status"] == ib["status"] == P.PAT_STATUS_CONVERGED
    assert ia["iters_done"] == ib["iters_done"] < 2000
    assert torch.equal(u_a, u_b)
    # at most 6 launches per iteration (3 + the gap's 3 every 10th) for the iterations run
    # plus two chunks of 8 periods of 10 iterations
    assert launches <= 6 * (ib["iters_done"] + 2 * 8 * 10 + 20) + 50


def test_tune_step_ratio_batched_equals_single_problem_tuning():
    ws = [make("small", seed=13 + k, reg=k % 2, beta=0.5) for k in range(3)]
    geos = [P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"]) for w in ws]
    fs = [dev(w["f"]) for w in ws]
    prms = [P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"]) for w in ws]
    cands = [0.5, 2.0, 8.0]
    best, gaps = P.pat_tune_step_ratio_batched([g.handle for g in geos], fs, prms, cands, 30)
    for k in range(3):
        b1, g1 = P.pat_tune_step_ratio(geos[k].handle, fs[k], prms[k], cands, 30)
        assert b1 == best[k] and g1 == gaps[k]


def test_disc64_tv_200_iterations():
    """The 64^2 TV disc reconstruction after its 200 iterations."""
    w = make("disc64", seed=0)
    pb = oracle_problem(w)
    ref = O.pdhg(pb, w["iters"], gap_every=50)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    prm = P.make_params(reg=0, alpha=w["alpha"], iters=w["iters"], gap_every=50)
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert rel_l2(host(u_d), ref.u) <= 1e-3
    assert abs(info["rel_gap"] - ref.gap["rel_gap"]) <= 1e-3 * max(ref.gap["rel_gap"], 1e-3)


@pytest.mark.parametrize("reg", [0, 1])
def test_scalar2_rule_parity(reg):
    w = make("small", seed=8, reg=reg, beta=0.5)
    pb = oracle_problem(w)
    ref = O.pdhg(pb, 40, steps=O.scalar2_steps(pb), gap_every=0)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    prm = P.make_params(reg=reg, alpha=w["alpha"], beta=w["beta"], iters=40, gap_every=0,
                        precond=P.PAT_PRECOND_SCALAR2)
    P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert rel_l2(host(u_d), ref.u) <= 1e-3


def test_tolerance_stop_matches_oracle():
    w = make("small", seed=9, reg=1, beta=0.5)
    pb = oracle_problem(w)
    tol = 2e-2
    ref = O.pdhg(pb, 2000, tol=tol, gap_every=5)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(w["n"], w["n"], device=DEV)
    prm = P.make_params(reg=1, alpha=w["alpha"], beta=w["beta"], iters=2000, tol=tol, gap_every=5)
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    assert ref.iters_done < 2000
    assert info["status"] == P.PAT_STATUS_CONVERGED
    assert abs(info["iters_done"] - ref.iters_done) <= 5
    assert info["rel_gap"] <= tol
    if info["iters_done"] == ref.iters_done:
        assert rel_l2(host(u_d), ref.u) <= 1e-3


@pytest.mark.parametrize("reg", [0, 1, 2])
def test_resume_from_exported_state_is_bit_exact(reg):
    """A run of 40 iterations equals, bit for bit, a run of 25 whose exported state (high
    and low words of the compensated primal pairs, xbar, y) starts a run of 15."""
    w = make("small", seed=10, reg=reg, beta=0.5)
    n = w["n"]
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    f = dev(w["f"])
    xi = dev(w["xi"]) if reg == 2 else None
    nx = (3 if reg == 1 else 1) * n * n
    ny = w["f"].size + (5 if reg == 1 else 2) * n * n

    def run(iters, **kw):
        out = {k: torch.full((m,), float("nan"), device=DEV) for k, m in
               (("x", nx), ("xlo", nx), ("xbar", nx), ("y", ny))}
        u = torch.empty(n, n, device=DEV)
        P.pat_reconstruct(pg.handle, f, P.make_params(reg=reg, alpha=w["alpha"], beta=0.5, xi=xi, iters=iters,
                                                      gap_every=0, x_out=out["x"], x_lo_out=out["xlo"],
                                                      xbar_out=out["xbar"], y_out=out["y"], **kw), u)
        out["u"] = u
        return out

    full = run(40)
    half = run(25)
    rest = run(15, x0=half["x"], x_lo0=half["xlo"], xbar0=half["xbar"], y0=half["y"])
    for k in ("u", "x", "xlo", "xbar", "y"):
        assert torch.equal(rest[k], full[k]), k
    assert torch.count_nonzero(full["xlo"]) > 0   # the low words carry information


def test_zero_iterations_returns_start():
    w = make("small", seed=1)
    n = w["n"]
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    x0 = np.random.default_rng(0).uniform(size=n * n).astype(np.float32)
    u_d = torch.zeros(n, n, device=DEV)
    x0d = dev(x0)
    info = P.pat_reconstruct(pg.handle, dev(w["f"]), P.make_params(iters=0, x0=x0d), u_d)
    assert info["iters_done"] == 0
    assert np.array_equal(host(u_d).ravel(), x0.astype(np.float64))


def test_direction_field_parity():
    n = 40
    wimg = S.side_image(n, 3).astype(np.float32)
    eta = 0.02
    xi_d = torch.empty(2, n, n, device=DEV)
    P.pat_direction_field(n, dev(wimg), eta, xi_d)
    ref = O.direction_field(wimg.astype(np.float64), eta)
    assert rel_l2(host(xi_d), ref) <= 1e-5


def test_invalid_arguments_and_nonfinite_data():
    w = make("small", seed=1)
    n = w["n"]
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    u_d = torch.empty(n, n, device=DEV)
    f = dev(w["f"])
    for bad in (dict(reg=7), dict(alpha=-1.0), dict(theta=1.5), dict(reg=2), dict(box_u=0.0), dict(iters=-1)):
        with pytest.raises(P.PatError) as ei:
            P.pat_reconstruct(pg.handle, f, P.make_params(**bad), u_d)
        assert ei.value.code == P.PAT_ERR_INVALID_ARG
    fbad = w["f"].copy()
    fbad[0, 0] = np.nan
    with pytest.raises(P.PatError) as ei:
        P.pat_reconstruct(pg.handle, dev(fbad), P.make_params(iters=20, gap_every=10), u_d)
    assert ei.value.code == P.PAT_ERR_NONFINITE
    # the context stays usable
    info = P.pat_reconstruct(pg.handle, f, P.make_params(iters=5), u_d)
    assert info["iters_done"] == 5


def test_full_size_tgv_one_iteration_from_state():
    """The 256^2 TGV workload (256 detectors x 512 samples): one iteration from a random
    state, in the launch configuration of the benchmark, against the matrix-free oracle."""
    w = make("tgv256", seed=0)
    n, S_ = w["n"], w["f"].size
    pb = oracle_problem(w, matrix=False)
    st = _random_state(w, 1, np.random.default_rng(3), scale=0.05)
    f32 = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)  # noqa: E731
    ref = O.pdhg(pb, 1, x0={"u": f32(st["u"]), "v": f32(st["v"])},
                 y0={"q": f32(st["q"]), "r": f32(st["r"]), "s": f32(st["s"])},
                 xbar0={"u": f32(st["ub"]), "v": f32(st["vb"])})
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    xo, yo = torch.empty(st["x"].size, device=DEV), torch.empty(st["y"].size, device=DEV)
    u_d = torch.empty(n, n, device=DEV)
    prm = P.make_params(reg=1, alpha=w["alpha"], beta=w["beta"], iters=1, gap_every=0, x0=dev(st["x"]),
                        xbar0=dev(st["xb"]), y0=dev(st["y"]), x_out=xo, y_out=yo)
    P.pat_reconstruct(pg.handle, dev(w["f"]), prm, u_d)
    xg, yg = host(xo), host(yo)
    assert rel_l2(xg[:n * n], ref.u) <= 1e-5
    assert rel_l2(yg[:S_], ref.q) <= 1e-5
    assert rel_l2(xg[n * n:], ref.v) <= 1e-5
    assert rel_l2(yg[S_ + 2 * n * n:], ref.s) <= 1e-5


def _batch_problem(name, seed, reg, **over):
    w = make(name, seed=seed, reg=reg, **over)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    return w, pg


def test_batched_matches_single_runs_bitwise():
    """Problems of different sizes and regularisers in one lockstep batch give exactly the
    iterates of their single runs (every kernel is deterministic)."""
    specs = [("small", 1, 0, {}), ("small", 2, 1, {"beta": 0.5}), ("small", 3, 2, {}),
             ("small", 4, 1, {"beta": 0.3, "n": 20})]
    probs = []
    for name, seed, reg, over in specs:
        if "n" in over:
            w = S.workload(name, seed)
            w.update(over)
            w["n_fine"] = 2 * w["n"]
            w["phantom_fine"] = S.rasterise_discs(S.disc_params(3, seed), 2 * w["n"])
            from tests.problems import noisy_data
            w["f"] = noisy_data(w)
            w["reg"], w["beta"] = reg, over["beta"]
            pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
        else:
            w, pg = _batch_problem(name, seed, reg, **over)
        probs.append((w, pg))
    iters = 45
    singles, fs, xis, prms, outs = [], [], [], [], []
    for w, pg in probs:
        f = dev(w["f"])
        xi = dev(w["xi"]) if w["reg"] == 2 else None
        u = torch.empty(w["n"], w["n"], device=DEV)
        prm = P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi, iters=iters,
                            gap_every=10)
        P.pat_reconstruct(pg.handle, f, prm, u)
        singles.append(host(u))
        fs.append(f)
        xis.append(xi)
        prms.append(prm)
        outs.append(torch.zeros(w["n"], w["n"], device=DEV))
    infos = P.pat_reconstruct_batched([pg.handle for _, pg in probs], fs, prms, outs)
    for (w, _), s_u, o, inf in zip(probs, singles, outs, infos):
        assert inf["iters_done"] == iters
        assert np.array_equal(host(o), s_u)


def test_batched_groups_unequal_iteration_counts():
    w1, g1 = _batch_problem("small", 5, 0)
    w2, g2 = _batch_problem("small", 6, 1, beta=0.5)
    f1, f2 = dev(w1["f"]), dev(w2["f"])
    p1 = P.make_params(reg=0, alpha=w1["alpha"], iters=12, gap_every=4)
    p2 = P.make_params(reg=1, alpha=w2["alpha"], beta=0.5, iters=30, gap_every=10)
    o1, o2 = torch.empty(w1["n"], w1["n"], device=DEV), torch.empty(w2["n"], w2["n"], device=DEV)
    infos = P.pat_reconstruct_batched([g1.handle, g2.handle], [f1, f2], [p1, p2], [o1, o2])
    assert [i["iters_done"] for i in infos] == [12, 30]
    s1 = torch.empty_like(o1)
    P.pat_reconstruct(g1.handle, f1, P.make_params(reg=0, alpha=w1["alpha"], iters=12, gap_every=4), s1)
    assert np.array_equal(host(o1), host(s1))


def test_graph_replay_matches_direct_launches():
    """The periodic part of the loop is replayed from a CUDA graph; with the profiler on the
    same iterations run as direct launches.  Both give identical iterates."""
    w, pg = _batch_problem("small", 7, 1, beta=0.5)
    f = dev(w["f"])
    prm = P.make_params(reg=1, alpha=w["alpha"], beta=0.5, iters=57, gap_every=5)
    u_graph, u_direct = torch.empty(w["n"], w["n"], device=DEV), torch.empty(w["n"], w["n"], device=DEV)
    P.pat_reconstruct(pg.handle, f, prm, u_graph)   # first call also computes the K sums
    n0 = P.pat_kernel_launches()
    P.pat_reconstruct(pg.handle, f, prm, u_graph)
    n_graph = P.pat_kernel_launches() - n0
    P.pat_profile_enable(True)
    try:
        n0 = P.pat_kernel_launches()
        P.pat_reconstruct(pg.handle, f, prm, u_direct)
        n_direct = P.pat_kernel_launches() - n0
    finally:
        P.pat_profile_enable(False)
        P.pat_profile_read(reset=True)
    assert np.array_equal(host(u_graph), host(u_direct))
    assert n_graph == n_direct
