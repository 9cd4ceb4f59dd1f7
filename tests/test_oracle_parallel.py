"""The process-parallel harness of the oracle (detector subsets on worker processes)
returns the oracle's own K, K^T and sampled rows (up to FP64 summation order)."""
import numpy as np

import synthetic as S
from oracle import pat_oracle as O
from oracle.parallel import OraclePool


def test_pool_matches_single_process_oracle():
    g = O.Geometry(n=20, det_xy=S.detectors_full_circle(9, 1.2), n_t=30, r0=0.0, dr=2.62 / 30, quad_m=48)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((20, 20))
    y = rng.standard_normal((9, 30))
    with OraclePool(g, workers=3) as pool:
        assert len(pool.spans) == 3 and pool.spans[0][0] == 0 and pool.spans[-1][1] == 9
        np.testing.assert_array_equal(pool.forward(u), O.forward(g, u))
        np.testing.assert_allclose(pool.adjoint(y), O.adjoint(g, y), rtol=1e-13, atol=1e-13)
        rows = np.array([0, 7, 31, 100, 269])
        np.testing.assert_allclose(pool.forward_rows(u, rows), O.forward(g, u).ravel()[rows], rtol=1e-13)
        pb = pool.problem(O.forward(g, u).ravel(), reg=O.REG_TV, alpha=0.05)
        ref = O.problem_from_geometry(g, O.forward(g, u).ravel(), reg=O.REG_TV, alpha=0.05)
        a = O.pdhg(pb, 5, gap_every=0, final_gap=False)
        b = O.pdhg(ref, 5, gap_every=0, final_gap=False)
        np.testing.assert_allclose(a.u, b.u, rtol=1e-11, atol=1e-13)


def test_pool_with_one_worker_runs_in_process():
    g = O.Geometry(n=8, det_xy=S.detectors_full_circle(2, 1.2), n_t=6, r0=0.0, dr=0.4, quad_m=16)
    pool = OraclePool(g, workers=1)
    assert pool.pool is None
    u = np.ones((8, 8))
    np.testing.assert_array_equal(pool.forward(u), O.forward(g, u))
    pool.close()
