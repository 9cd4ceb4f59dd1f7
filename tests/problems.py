"""Test-side construction of reconstruction problems from the seeded workload recipes.

Data are simulated with the FP64 oracle on the 2x finer grid (inverse-crime avoidance,
Sec. 5.2) and perturbed with the recipe's Gaussian noise; the same float32 data feed
both the CUDA path and the oracle in every parity test.
"""
import numpy as np

import synthetic as S
from oracle import pat_oracle as O


def oracle_geometry(w, fine=False):
    return O.Geometry(n=w["n_fine"] if fine else w["n"], det_xy=w["det_xy"], n_t=w["n_t"], r0=w["r0"],
                      dr=w["dr"], quad_m=w["quad_m_fine"] if fine else w["quad_m"])


def noisy_data(w):
    clean = O.forward(oracle_geometry(w, fine=True), w["phantom_fine"])
    return (clean + w["noise_level"] * np.abs(clean).max() * w["noise"]).astype(np.float32)


def direction_field32(w):
    return O.direction_field(w["side"], w["eta"]).astype(np.float32)


def make(name, seed=0, **over):
    w = S.workload(name, seed)
    w.update(over)
    w["f"] = noisy_data(w)
    if w["reg"] == O.REG_DTV:
        if "side" not in w:
            w["side"] = S.side_image(w["n"], seed)
            w["eta"] = 0.01 * float(w["side"].max() - w["side"].min())
        w["xi"] = direction_field32(w)
    return w


def oracle_problem(w, reg=None, matrix=True, **kw):
    reg = w["reg"] if reg is None else reg
    g = oracle_geometry(w)
    args = dict(reg=reg, alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"],
                xi=w.get("xi").astype(np.float64) if w.get("xi") is not None else None)
    args.update(kw)
    f = w["f"].astype(np.float64)
    if matrix:
        return O.problem_from_geometry(g, f, **args)
    n = g.n
    krow = O.forward(g, np.ones((n, n))).ravel()
    kcol = O.adjoint(g, np.ones((g.n_det, g.n_t)))
    return O.Problem(n=n, K=lambda u: O.forward(g, u).ravel(), KT=lambda y: O.adjoint(g, y), f=f,
                     k_abs_rows=krow, k_abs_cols=kcol, **args)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
