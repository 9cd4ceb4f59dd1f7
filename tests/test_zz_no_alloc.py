"""pat_adjoint_noalloc: K^T for callers that cannot allocate device memory during the call
(for example code running under CUDA graph capture, or applications whose device memory
belongs to another allocator).  Its scratch is a device array built into the library, so
the test checks two calls in a row against pat_adjoint, which allocates its own scratch.

This file sorts last so that a run stopping at the first failure has already run every
other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1707_02245_gb300 as P  # noqa: E402
from paper_1707_02245_gb300 import build as B  # noqa: E402

DEV = torch.device("cuda:0")


def _rel(a, b):
    a = a.detach().cpu().double().ravel()
    b = b.detach().cpu().double().ravel()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.fixture(scope="module")
def geometry():
    B.build()
    P.load()
    w = S.workload("tgv256")
    g = P.Geometry(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    yield w, g
    g.close()


def test_noalloc_adjoint_matches_pat_adjoint_on_two_calls(geometry):
    w, g = geometry
    n, d, t = w["n"], w["det_xy"].shape[0], w["n_t"]
    rng = np.random.default_rng(5)
    y1 = torch.from_numpy(rng.standard_normal((d, t)).astype(np.float32)).to(DEV)
    y2 = torch.from_numpy((0.01 * rng.standard_normal((d, t))).astype(np.float32)).to(DEV)
    ref1 = torch.empty(n, n, device=DEV)
    ref2 = torch.empty(n, n, device=DEV)
    # pat_adjoint prepares the geometry (FP64 K sums) while allocation is allowed
    P.pat_adjoint(g.handle, y1, ref1)
    P.pat_adjoint(g.handle, y2, ref2)
    out1 = torch.full((n, n), float("nan"), device=DEV)
    out2 = torch.full((n, n), float("nan"), device=DEV)
    P.pat_adjoint_noalloc(g.handle, y1, out1)
    P.pat_adjoint_noalloc(g.handle, y2, out2)   # second call: the scratch holds the first call's state
    torch.cuda.synchronize()
    assert torch.isfinite(out1).all() and torch.isfinite(out2).all()
    assert _rel(out1, ref1) <= 1e-6
    assert _rel(out2, ref2) <= 1e-6


def test_noalloc_adjoint_rejects_oversized_and_unprepared_geometry():
    B.build()
    P.load()
    big = P.Geometry(1025, np.array([[1.5, 0.0]]), 4, 0.0, 0.5, 8)
    y = torch.zeros(1, 4, device=DEV)
    u = torch.empty(1025, 1025, device=DEV)
    with pytest.raises(P.PatError) as ei:
        P.pat_adjoint_noalloc(big.handle, y, u)
    assert ei.value.code == P.PAT_ERR_INVALID_ARG and "1024" in str(ei.value)
    big.close()
    fresh = P.Geometry(16, np.array([[1.5, 0.0]]), 8, 0.0, 0.4, 16)
    with pytest.raises(P.PatError) as ei:
        P.pat_adjoint_noalloc(fresh.handle, torch.zeros(1, 8, device=DEV), torch.empty(16, 16, device=DEV))
    assert ei.value.code == P.PAT_ERR_INVALID_ARG and "prepared" in str(ei.value)
    fresh.close()
