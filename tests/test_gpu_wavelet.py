"""Parity of the wavelet model (PAT_WAV, Sec. 2.2 eq. (min_wav)) with the FP64 oracle:
the transform and its transpose (rel 1e-6), the diagonal steps (rel-L2 1e-5), and the
image after a fixed number of PDHG iterations (rel-L2 1e-3, the stated target), with the
gap to 1e-4 of the primal value."""
import numpy as np
import pytest

import synthetic as S
from oracle import pat_oracle as O
from oracle import wavelet_oracle as WO
from tests.problems import noisy_data

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


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("n,levels", [(16, 1), (16, 4), (24, 3), (64, 4), (256, 5)])
def test_transform_and_transpose_match_oracle(n, levels):
    rng = np.random.default_rng(n + levels)
    u = rng.standard_normal((n, n)).astype(np.float32)
    out = torch.empty(n, n, device=DEV)
    P.pat_wavelet_transform(n, levels, dev(u), out)
    ref = WO.dwt2(u.astype(np.float64), levels)
    assert rel_l2(host(out), ref) < 1e-6
    back = torch.empty(n, n, device=DEV)
    P.pat_wavelet_transform(n, levels, out, back, inverse=True)
    assert rel_l2(host(back), WO.idwt2(host(out), levels)) < 1e-6
    assert rel_l2(host(back), u) < 1e-6


def _geom(n=16, n_det=10, n_t=24, m=48):
    det = S.detectors_full_circle(n_det, 1.2)
    r0, dr = S.radial_sampling(det, n_t)
    return dict(n=n, det_xy=det, n_t=n_t, r0=r0, dr=dr, quad_m=m, n_fine=2 * n, quad_m_fine=2 * m)


def _problem(seed=0, n=16, levels=2, alpha=0.02):
    w = _geom(n=n)
    discs = S.disc_params(3, seed)
    w["phantom_fine"] = S.rasterise_discs(discs, 2 * n)
    w["noise"] = S.standard_normal((w["det_xy"].shape[0], w["n_t"]), seed + 17)
    w["noise_level"] = 0.02
    f = noisy_data(w)
    og = O.Geometry(n=n, det_xy=w["det_xy"], n_t=w["n_t"], r0=w["r0"], dr=w["dr"], quad_m=w["quad_m"])
    Km = O.system_matrix(og)
    pg = P.Geometry(n, w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    return w, f, og, Km, pg


def test_wavelet_steps_match_oracle():
    w, f, og, Km, pg = _problem()
    n, levels = w["n"], 2
    krow = np.asarray(abs(Km).sum(axis=1)).ravel()
    kcol = np.asarray(abs(Km).sum(axis=0)).ravel()
    sq, sr, tu = WO.wavelet_steps(kcol, krow, n, levels)
    prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, wavelet_levels=levels)
    a = torch.empty(f.size, device=DEV)
    b = torch.empty(n, n, device=DEV)
    c = torch.empty(n, n, device=DEV)
    P.pat_steps(pg.handle, prm, sig_q=a, tau_u=b, sig_r=c)
    assert rel_l2(host(a), sq) < 1e-5
    assert rel_l2(host(b), tu) < 1e-5
    assert rel_l2(host(c), sr) < 1e-5


@pytest.mark.parametrize("ratio", [1.0, 3.0])
def test_wavelet_pdhg_fixed_iterations_match_oracle(ratio):
    w, f, og, Km, pg = _problem(seed=1)
    n, levels, alpha, iters = w["n"], 2, 0.02, 120
    krow = np.asarray(abs(Km).sum(axis=1)).ravel()
    kcol = np.asarray(abs(Km).sum(axis=0)).ravel()
    sq, sr, tu = WO.wavelet_steps(kcol, krow, n, levels)
    Kf = lambda u: Km @ np.ravel(u)
    KTf = lambda q: Km.T @ q
    u_ref, q_ref, r_ref, hist = WO.pdhg_wavelet(Kf, KTf, f.astype(np.float64), n, levels, alpha, iters, sq, sr, tu,
                                                gap_every=40, step_ratio=ratio)
    u_d = torch.empty(n, n, device=DEV)
    y_d = torch.empty(f.size + n * n, device=DEV)
    prm = P.make_params(reg=P.PAT_WAV, alpha=alpha, iters=iters, gap_every=40, wavelet_levels=levels,
                        step_ratio=ratio, y_out=y_d)
    info = P.pat_reconstruct(pg.handle, dev(f), prm, u_d)
    assert info["iters_done"] == iters
    assert rel_l2(host(u_d), u_ref) <= 1e-3
    assert rel_l2(host(y_d)[f.size:], r_ref.ravel()) <= 1e-3
    gap_ref = hist[-1][1]
    prim = WO.wavelet_gap(Kf, KTf, f, n, levels, alpha, u_ref, q_ref, r_ref)["primal"]
    assert abs(info["gap"] - gap_ref) <= 1e-4 * prim


def test_wavelet_tolerance_stop_and_long_cap():
    w, f, og, Km, pg = _problem(seed=2)
    n = w["n"]
    u_d = torch.empty(n, n, device=DEV)
    prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=200000, tol=1e-3, gap_every=10, wavelet_levels=2)
    l0 = P.pat_kernel_launches()
    info = P.pat_reconstruct(pg.handle, dev(f), prm, u_d)
    launches = P.pat_kernel_launches() - l0
    assert info["status"] == P.PAT_STATUS_CONVERGED and info["rel_gap"] <= 1e-3
    assert info["iters_done"] % 10 == 0
    # replays end soon after the stop (far fewer launches than 200000 iterations)
    assert launches < 40 * (info["iters_done"] + 200)
    with pytest.raises(P.PatError):
        P.pat_reconstruct(pg.handle, dev(f), P.make_params(reg=P.PAT_WAV, alpha=0.02, wavelet_levels=5), u_d)
