"""Parity of the dual-tree complex wavelet transform (Sec. 2.2) and of the wavelet model with
it (PAT_WAV, wavelet_kind = PAT_WAVELET_DTCWT) with the FP64 oracle
(oracle/dtcwt_oracle.py): W and W^T (rel 1e-6), the diagonal steps (rel-L2 1e-5), and the
image after a fixed number of PDHG iterations (rel-L2 1e-3, the stated target), with the
gap to 1e-4 of the primal value."""
import numpy as np
import pytest

import synthetic as S
from oracle import dtcwt_oracle as D
from oracle import pat_oracle as O
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
    rng = np.random.default_rng(n + 3 * levels)
    u = rng.standard_normal((n, n)).astype(np.float32)
    out = torch.empty(4, n, n, device=DEV)
    P.pat_dtcwt_transform(n, levels, dev(u), out)
    ref = D.dtcwt2(u.astype(np.float64), levels)
    assert rel_l2(host(out), ref) < 1e-6
    c = rng.standard_normal((4, n, n)).astype(np.float32)
    back = torch.empty(n, n, device=DEV)
    P.pat_dtcwt_transform(n, levels, dev(c), back, inverse=True)
    assert rel_l2(host(back), D.idtcwt2(c.astype(np.float64), levels)) < 1e-6
    P.pat_dtcwt_transform(n, levels, out, back, inverse=True)
    assert rel_l2(host(back), u) < 1e-6      # W^T W = I


def test_custom_filters_match_oracle():
    # any orthonormal pair: the one-angle lattice filter with theta = 0.3 at level 1, and
    # the Daubechies filter as the Q-shift filter
    c, s_ = np.cos(0.3), np.sin(0.3)
    hl = np.array([1 - c + s_, 1 + c + s_, 1 + c - s_, 1 - c - s_]) / (2 * np.sqrt(2.0))
    filters = (hl, D.D4)
    n, levels = 32, 3
    u = np.random.default_rng(5).standard_normal((n, n)).astype(np.float32)
    out = torch.empty(4, n, n, device=DEV)
    P.pat_dtcwt_transform(n, levels, dev(u), out, filters=filters)
    assert rel_l2(host(out), D.dtcwt2(u.astype(np.float64), levels, filters)) < 1e-6


def test_bad_filters_are_rejected():
    u = torch.zeros(16, 16, device=DEV)
    out = torch.empty(4, 16, 16, device=DEV)
    with pytest.raises(P.PatError):
        P.pat_dtcwt_transform(16, 2, u, out, filters=(np.array([1.0, 1.0, 0.0]), D.QSHIFT4))   # odd length
    with pytest.raises(P.PatError):
        P.pat_dtcwt_transform(16, 2, u, out, filters=(D.D4, np.array([0.5, 0.5, 0.5, 0.5])))   # not orthonormal


def _problem(seed=0, n=16):
    det = S.detectors_full_circle(10, 1.2)
    r0, dr = S.radial_sampling(det, 24)
    w = dict(n=n, det_xy=det, n_t=24, r0=r0, dr=dr, quad_m=48, n_fine=2 * n, quad_m_fine=96)
    w["phantom_fine"] = S.rasterise_discs(S.disc_params(3, seed), 2 * n)
    w["noise"] = S.standard_normal((10, 24), seed + 17)
    w["noise_level"] = 0.02
    f = noisy_data(w)
    og = O.Geometry(n=n, det_xy=det, n_t=24, r0=r0, dr=dr, quad_m=48)
    Km = O.system_matrix(og)
    pg = P.Geometry(n, det, 24, r0, dr, 48)
    return w, f, Km, pg


def test_dtcwt_steps_match_oracle():
    w, f, Km, pg = _problem()
    n, levels = w["n"], 2
    krow = np.asarray(abs(Km).sum(axis=1)).ravel()
    kcol = np.asarray(abs(Km).sum(axis=0)).ravel()
    sq, sr, tu = D.cwt_steps(kcol, krow, n, levels)
    prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, wavelet_levels=levels, wavelet_kind=P.PAT_WAVELET_DTCWT)
    a = torch.empty(f.size, device=DEV)
    b = torch.empty(n, n, device=DEV)
    c = torch.empty(4, n, n, device=DEV)
    P.pat_steps(pg.handle, prm, sig_q=a, tau_u=b, sig_r=c)
    assert rel_l2(host(a), sq) < 1e-5
    assert rel_l2(host(b), tu) < 1e-5
    assert rel_l2(host(c), sr) < 1e-5
    pg.close()


@pytest.mark.parametrize("ratio", [1.0, 3.0])
def test_dtcwt_pdhg_fixed_iterations_match_oracle(ratio):
    w, f, Km, pg = _problem(seed=1)
    n, levels, alpha, iters = w["n"], 2, 0.02, 120
    krow = np.asarray(abs(Km).sum(axis=1)).ravel()
    kcol = np.asarray(abs(Km).sum(axis=0)).ravel()
    sq, sr, tu = D.cwt_steps(kcol, krow, n, levels)
    Kf = lambda u: Km @ np.ravel(u)
    KTf = lambda q: Km.T @ q
    u_ref, q_ref, r_ref, hist = D.pdhg_cwt(Kf, KTf, f.astype(np.float64), n, levels, alpha, iters, sq, sr, tu,
                                           gap_every=40, step_ratio=ratio)
    u_d = torch.empty(n, n, device=DEV)
    y_d = torch.empty(f.size + 4 * n * n, device=DEV)
    prm = P.make_params(reg=P.PAT_WAV, alpha=alpha, iters=iters, gap_every=40, wavelet_levels=levels,
                        wavelet_kind=P.PAT_WAVELET_DTCWT, step_ratio=ratio, y_out=y_d)
    info = P.pat_reconstruct(pg.handle, dev(f), prm, u_d)
    assert info["iters_done"] == iters
    assert rel_l2(host(u_d), u_ref) <= 1e-3
    assert rel_l2(host(y_d)[f.size:], r_ref.ravel()) <= 1e-3
    prim = D.cwt_gap(Kf, KTf, f, n, levels, alpha, u_ref, q_ref, r_ref)["primal"]
    assert abs(info["gap"] - hist[-1][1]) <= 1e-4 * prim
    pg.close()


def test_dtcwt_model_at_benchmark_size_reaches_tolerance():
    """The DT-CWT model on a 256^2 benchmark-size geometry (128 detectors, T = 512, data of
    a vessel phantom with 2% noise) stops at rel_gap 1e-3 within its cap."""
    w = S.workload_warm(11, n=256, n_det=128)
    pg = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    clean = torch.empty(128, w["n_t"], device=DEV)
    P.pat_forward(pg.handle, dev(S.vessel_phantom(256, 11)), clean)
    noise = dev(S.standard_normal((128, w["n_t"]), 5))
    f = (clean + 0.02 * clean.abs().max() * noise).contiguous()
    u_d = torch.empty(256, 256, device=DEV)
    prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=20000, tol=1e-3, gap_every=20, wavelet_levels=4,
                        wavelet_kind=P.PAT_WAVELET_DTCWT)
    info = P.pat_reconstruct(pg.handle, f, prm, u_d)
    assert info["status"] == P.PAT_STATUS_CONVERGED and info["rel_gap"] <= 1e-3
    assert np.isfinite(host(u_d)).all()
    pg.close()


def _problem_det(seed, n_det, n=16):
    det = S.detectors_full_circle(n_det, 1.2)
    r0, dr = S.radial_sampling(det, 24)
    w = dict(n=n, det_xy=det, n_t=24, r0=r0, dr=dr, quad_m=48, n_fine=2 * n, quad_m_fine=96)
    w["phantom_fine"] = S.rasterise_discs(S.disc_params(3, seed), 2 * n)
    w["noise"] = S.standard_normal((n_det, 24), seed + 17)
    w["noise_level"] = 0.02
    return noisy_data(w), P.Geometry(n, det, 24, r0, dr, 48)


@pytest.mark.parametrize("kind", [P.PAT_WAVELET_DWT, P.PAT_WAVELET_DTCWT])
def test_wavelet_batch_gives_the_single_runs_bits(kind):
    """Wavelet problems of one N and transform run as one lockstep batch (K, K^T and every
    wavelet kernel launch once for all of them, each problem's buffers a fixed stride apart)
    and give each problem's single-run image, dual state and gap bit for bit.  The batch mixes
    geometries (10 and 12 detectors), alpha, theta and tolerances: the third problem meets its
    tolerance (relative gap 2, near iteration 80 or 90 with a gap evaluation every 10) and stops while the
    others go on.  A 32^2 wavelet problem and a TV problem in the same call run in batches
    of their own."""
    iters = 120
    specs = [(1, 10, 16, 0.02, 1.0, 0.0), (2, 12, 16, 0.05, 0.8, 0.0), (3, 10, 16, 0.02, 1.0, 2.0),
             (4, 10, 32, 0.03, 1.0, 0.0)]
    probs = []
    for seed, n_det, n, alpha, theta, tol in specs:
        f, pg = _problem_det(seed, n_det, n)
        fd = dev(f)
        y = torch.zeros(f.size + 4 * n * n, device=DEV)
        prm = P.make_params(reg=P.PAT_WAV, alpha=alpha, theta=theta, tol=tol, iters=iters, gap_every=10,
                            wavelet_levels=2, wavelet_kind=kind, y_out=y)
        u = torch.empty(n, n, device=DEV)
        info = P.pat_reconstruct(pg.handle, fd, prm, u)
        probs.append(dict(pg=pg, f=fd, n=n, u=host(u), y=host(y), info=info, tol=tol, alpha=alpha, theta=theta,
                          kind=kind))
    assert probs[2]["info"]["iters_done"] < iters and probs[0]["info"]["iters_done"] == iters
    # a TV problem in the same call
    ft, pt = _problem_det(5, 10, 16)
    ftd = dev(ft)
    ptv = P.make_params(reg=P.PAT_TV, alpha=0.02, iters=iters, gap_every=10)
    ut = torch.empty(16, 16, device=DEV)
    P.pat_reconstruct(pt.handle, ftd, ptv, ut)
    ut_single = host(ut)
    outs, ys, prms = [], [], []
    for q in probs:
        n = q["n"]
        outs.append(torch.zeros(n, n, device=DEV))
        ys.append(torch.zeros(q["y"].size, device=DEV))
        prms.append(P.make_params(reg=P.PAT_WAV, alpha=q["alpha"], theta=q["theta"], tol=q["tol"], iters=iters,
                                  gap_every=10, wavelet_levels=2, wavelet_kind=kind, y_out=ys[-1]))
    ut_b = torch.zeros(16, 16, device=DEV)
    infos = P.pat_reconstruct_batched([q["pg"].handle for q in probs] + [pt.handle], [q["f"] for q in probs] + [ftd],
                                      prms + [ptv], outs + [ut_b])
    for q, o, y, inf in zip(probs, outs, ys, infos):
        assert inf["iters_done"] == q["info"]["iters_done"] and inf["status"] == q["info"]["status"]
        assert np.array_equal(host(o), q["u"])
        assert np.array_equal(host(y), q["y"])
        assert inf["gap"] == q["info"]["gap"] and inf["rel_gap"] == q["info"]["rel_gap"]
    assert np.array_equal(host(ut_b), ut_single)
    for q in probs:
        q["pg"].close()
    pt.close()


def test_wavelet_step_ratio_probes_run_as_one_batch():
    """The balance probes of a wavelet problem run as one batch of candidates; each probe's
    relative gap equals that of a single run with the candidate's step ratio."""
    f, pg = _problem_det(1, 10, 16)
    fd = dev(f)
    prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=100, gap_every=10, wavelet_levels=2,
                        wavelet_kind=P.PAT_WAVELET_DTCWT)
    cands = [0.5, 1.0, 4.0]
    best, gaps = P.pat_tune_step_ratio(pg.handle, fd, prm, cands, 30)
    u = torch.empty(16, 16, device=DEV)
    for c, gq in zip(cands, gaps):
        q = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=30, gap_every=0, wavelet_levels=2,
                          wavelet_kind=P.PAT_WAVELET_DTCWT, step_ratio=c)
        assert P.pat_reconstruct(pg.handle, fd, q, u)["rel_gap"] == gq
    assert best == cands[int(np.argmin(gaps))]
    pg.close()
