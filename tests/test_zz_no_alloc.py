"""pat_adjoint_noalloc: K^T for callers that cannot allocate device memory when they call
(for example a real-time loop whose device memory is fixed at start-up, or an application
whose device memory belongs to another allocator).  Its scratch is a device array built
into the library, so the test checks calls in a row against pat_adjoint, which allocates
its own scratch: two calls on one geometry, then a call on a smaller geometry (which must
not see the larger image the scratch still holds).  It also checks that the calls take
nothing from the device's stream-ordered memory pool.

This file sorts last so that a run stopping at the first failure has already run every
other test; it also passes alone in a fresh process.
"""
import ctypes

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


class _DefaultPool:
    """Used-memory counters of the current device's default stream-ordered pool, read with
    the driver API (every CUDA runtime in the process allocates from this pool)."""
    USED_CURRENT, USED_HIGH = 7, 8     # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)   # setting the high-water mark to 0 resets it to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(zero)) == 0


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
    # a smaller geometry, prepared the same way, for a third call after the large ones
    small_det = S.detectors_full_circle(24, 1.2)
    r0, dr = S.radial_sampling(small_det, 128)
    gs = P.Geometry(64, small_det, 128, r0, dr, 128)
    y3 = torch.from_numpy(rng.standard_normal((24, 128)).astype(np.float32)).to(DEV)
    ref3 = torch.empty(64, 64, device=DEV)
    P.pat_adjoint(gs.handle, y3, ref3)
    out1 = torch.full((n, n), float("nan"), device=DEV)
    out2 = torch.full((n, n), float("nan"), device=DEV)
    out3 = torch.full((64, 64), float("nan"), device=DEV)
    # the set-up call: the first call on a device looks up the scratch's address (and
    # loading the library's module places the scratch array in device memory)
    P.pat_adjoint_noalloc(gs.handle, y3, out3)
    torch.cuda.synchronize()
    out3.fill_(float("nan"))
    torch.cuda.synchronize()
    pool = _DefaultPool()
    pool.reset_high()
    used0 = pool.get(pool.USED_CURRENT)
    free0 = torch.cuda.mem_get_info()[0]
    P.pat_adjoint_noalloc(g.handle, y1, out1)
    P.pat_adjoint_noalloc(g.handle, y2, out2)   # second call: the scratch holds the first call's state
    P.pat_adjoint_noalloc(gs.handle, y3, out3)  # smaller image after larger ones
    torch.cuda.synchronize()
    assert pool.get(pool.USED_HIGH) == used0, "the calls took memory from the stream-ordered pool"
    assert pool.get(pool.USED_CURRENT) == used0
    assert torch.cuda.mem_get_info()[0] == free0
    # the results are pat_adjoint's bit for bit (same kernels, integer fixed-point sums)
    assert torch.equal(out1, ref1)
    assert torch.equal(out2, ref2)
    assert torch.equal(out3, ref3)
    # positive control: pat_adjoint itself draws its scratch from that pool
    pool.reset_high()
    P.pat_adjoint(gs.handle, y3, ref3)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_HIGH) > used0
    gs.close()


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
