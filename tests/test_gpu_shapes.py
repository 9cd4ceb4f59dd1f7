"""Launch shapes and their autotuner (pat_geometry_set_shapes, pat_tune_shapes).

Every shape computes the same operators.  K^T work items accumulate in integers and the
fused update is pointwise, so their shapes give the same bits; K variants add a row's
points in different orders, so they agree to FP32 rounding.  The tuner's choice is
cached in a JSON file and applied again without timing.
"""
import json
import os

import numpy as np
import pytest

import synthetic as S
from tests.problems import make, rel_l2

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


def _problem(reg=1):
    """A 256^2 TGV problem (several slabs for the shared-memory K variants), 128 detectors."""
    w = S.workload_warm(5, n=256, n_det=128)
    rng = np.random.default_rng(3)
    f = (rng.standard_normal((w["det_xy"].shape[0], w["n_t"])) * 0.1).astype(np.float32)
    g = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    return w, g, dev(f), reg


def _run(g, f, w, reg, iters=12):
    n = w["n"]
    nx = (3 if reg == 1 else 1) * n * n
    ny = f.numel() + (5 if reg == 1 else 2) * n * n
    out = {k: torch.empty(m, device=DEV) for k, m in (("x", nx), ("xlo", nx), ("y", ny))}
    u = torch.empty(n, n, device=DEV)
    P.pat_reconstruct(g.handle, f, P.make_params(reg=reg, alpha=0.02, beta=0.04, iters=iters, gap_every=5,
                                                 x_out=out["x"], x_lo_out=out["xlo"], y_out=out["y"]), u)
    torch.cuda.synchronize()
    out["u"] = u
    return out


def test_adjoint_waves_and_update_tiles_give_the_same_bits():
    w, g, f, reg = _problem()
    ref = _run(g, f, w, reg)
    base = P.pat_geometry_get_shapes(g.handle)
    for waves, tile in ((2, P.PAT_UPD_32X4), (1, P.PAT_UPD_32X8), (1, P.PAT_UPD_64X4), (2, P.PAT_UPD_64X4)):
        P.pat_geometry_set_shapes(g.handle, base["forward"], waves, tile)
        got = P.pat_geometry_get_shapes(g.handle)
        assert got["adjoint_waves"] == waves and got["update_tile"] == tile
        out = _run(g, f, w, reg)
        for k in ("u", "x", "xlo", "y"):
            assert torch.equal(out[k], ref[k]), (waves, tile, k)
    g.close()


def test_adjoint_waves_agree_on_ragged_geometries():
    """K^T alone with work items filling one to four waves, bit for bit, on geometries with
    short segments and ragged tiles (detectors inside the image, a limited arc, N and T
    not multiples of 32)."""
    rng = np.random.default_rng(12)
    cases = [(37, S.detectors_full_circle(20, 1.3), 61, 64),
             (50, np.array([[0.1, -0.2], [0.5, 0.4], [-0.9, 0.0]]), 45, 96),
             (96, S.detectors_full_circle(64, 1.2)[:20], 150, 128)]
    for n, det, n_t, m in cases:
        r0, dr = S.radial_sampling(det, n_t)
        g = P.Geometry(n, det, n_t, r0, dr, m)
        y = dev(rng.standard_normal((det.shape[0], n_t)))
        outs = []
        for waves in (1, 2, 3, 4):
            P.pat_geometry_set_shapes(g.handle, P.PAT_FWD_AUTO, waves, P.PAT_UPD_32X4)
            u = torch.empty(n, n, device=DEV)
            P.pat_adjoint(g.handle, y, u)
            outs.append(u)
        torch.cuda.synchronize()
        for o in outs[1:]:
            assert torch.equal(outs[0], o), n
        g.close()


@pytest.mark.parametrize("reg", [0, 1])
def test_forward_variants_agree(reg):
    w, g, f, _ = _problem(reg)
    outs = {}
    for fv in (P.PAT_FWD_SLAB_TWO, P.PAT_FWD_SLAB_ONE, P.PAT_FWD_GLOBAL):
        P.pat_geometry_set_shapes(g.handle, fv, 1, P.PAT_UPD_32X4)
        outs[fv] = (P.pat_geometry_get_shapes(g.handle)["forward"], _run(g, f, w, reg))
    assert outs[P.PAT_FWD_GLOBAL][0] == P.PAT_FWD_GLOBAL
    assert outs[P.PAT_FWD_SLAB_TWO][0] == P.PAT_FWD_SLAB_TWO
    ref = outs[P.PAT_FWD_GLOBAL][1]
    for fv, (_, out) in outs.items():
        assert rel_l2(out["u"].cpu().numpy(), ref["u"].cpu().numpy()) <= 1e-5, fv
    # K alone: every variant within FP32 rounding of the others
    rng = np.random.default_rng(8)
    u = dev(rng.standard_normal((w["n"], w["n"])))
    ys = []
    for fv in (P.PAT_FWD_SLAB_TWO, P.PAT_FWD_SLAB_ONE, P.PAT_FWD_GLOBAL):
        P.pat_geometry_set_shapes(g.handle, fv, 1, P.PAT_UPD_32X4)
        y = torch.empty(f.shape, device=DEV)
        P.pat_forward(g.handle, u, y)
        ys.append(y.cpu().numpy())
    for y in ys[1:]:
        assert rel_l2(y, ys[0]) <= 2e-6
    g.close()


def test_tuner_chooses_caches_and_reapplies(tmp_path):
    w, g, f, reg = _problem()
    prm = P.make_params(reg=reg, alpha=0.02, beta=0.04)
    cache = str(tmp_path / "shapes.json")
    chosen = P.pat_tune_shapes([g.handle], [f], [prm], reps=20, cache_path=cache)
    assert len(chosen) == 1 and chosen[0] == P.pat_geometry_get_shapes(g.handle)
    with open(cache) as fh:
        data = json.load(fh)
    (entry,) = data["entries"]
    assert "N=256 D=128 T=512 M=256 reg=1" in entry["key"]
    assert [entry["forward"], entry["adjoint_waves"], entry["update_tile"]] == \
        [chosen[0]["forward"], chosen[0]["adjoint_waves"], chosen[0]["update_tile"]]
    assert all(t > 0 for t in entry["us"])
    # a second geometry with the same key takes the cached shapes without timing
    g2 = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    P.pat_geometry_set_shapes(g2.handle, P.PAT_FWD_GLOBAL, 2, P.PAT_UPD_64X4)
    mtime = os.path.getmtime(cache)
    again = P.pat_tune_shapes([g2.handle], [f], [prm], reps=20, cache_path=cache)
    assert again == chosen
    assert os.path.getmtime(cache) == mtime
    # the tuned shapes reconstruct the same image as the default shapes (to FP32 rounding)
    ref = _run(g2, f, w, reg)
    P.pat_geometry_set_shapes(g2.handle, P.PAT_FWD_AUTO, 1, P.PAT_UPD_32X4)
    out = _run(g2, f, w, reg)
    assert rel_l2(out["u"].cpu().numpy(), ref["u"].cpu().numpy()) <= 1e-5
    g.close()
    g2.close()


def test_batch_of_mixed_shapes_equals_single_runs():
    """Problems whose geometries use different K variants and update tiles share a batch:
    each one's iterates equal its own single run bit for bit."""
    wa = make("small", seed=1, reg=1)
    wb = S.workload_warm(9, n=256, n_det=64)
    rng = np.random.default_rng(4)
    fb = (rng.standard_normal((64, wb["n_t"])) * 0.1).astype(np.float32)
    ga = P.Geometry(wa["n"], wa["det_xy"], wa["n_t"], wa["r0"], wa["dr"], wa["quad_m"])
    gb = P.Geometry(wb["n"], wb["det_xy"], wb["n_t"], wb["r0"], wb["dr"], wb["quad_m"])
    P.pat_geometry_set_shapes(ga.handle, P.PAT_FWD_GLOBAL, 1, P.PAT_UPD_32X8)
    P.pat_geometry_set_shapes(gb.handle, P.PAT_FWD_SLAB_TWO, 2, P.PAT_UPD_64X4)
    fa_d, fb_d = dev(wa["f"]), dev(fb)
    prm = [P.make_params(reg=1, alpha=0.05, beta=0.5, iters=30, gap_every=10),
           P.make_params(reg=1, alpha=0.02, beta=0.04, iters=30, gap_every=10)]
    ua, ub = torch.empty(wa["n"], wa["n"], device=DEV), torch.empty(256, 256, device=DEV)
    P.pat_reconstruct_batched([ga.handle, gb.handle], [fa_d, fb_d], prm, [ua, ub])
    sa, sb = torch.empty_like(ua), torch.empty_like(ub)
    P.pat_reconstruct(ga.handle, fa_d, prm[0], sa)
    P.pat_reconstruct(gb.handle, fb_d, prm[1], sb)
    torch.cuda.synchronize()
    assert torch.equal(ua, sa) and torch.equal(ub, sb)
    ga.close()
    gb.close()
