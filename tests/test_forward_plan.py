"""Host logic of the forward projector's work plan (pat_forward_plan; no GPU needed).

K runs as clusters of S CTAs: rank s stages image slab s in shared memory, and a cluster
owns a list of row groups (8 radii of one detector), processed in rounds of 256.  In a
round, each rank evaluates its units (a row group's points restricted to the rank's slab,
inside at most two angular windows, counting a point only when its upper-left tap row j0
lies in the slab and its tap column in the grid), then the ranks' partial sums are added.
So: every row group belongs to exactly one cluster; every quadrature point whose taps
touch the grid (Sec. 4.2, eq. (K_def)) lies inside a window of the unit of its row group
in the rank of its slab, in the round that holds the row group; a unit's two windows do
not overlap (a point would be counted twice); and a CTA's shared memory fits.  Checked by
brute force over every point (d, k, m) with the FP32 point arithmetic of the kernels.
"""
import math

import numpy as np
import pytest

import paper_1707_02245_gb300 as P
import synthetic as S

KGRP = 8


def _f32_points(n, det_xy, n_t, r0, dr, quad_m, extent=(-1.0, 1.0, -1.0, 1.0)):
    """(i0, j0) of every point (d, k, m) as the device computes them: fx = fmaf(r, cs.x, det.x)
    in FP32 (the exact product plus the addend, rounded once), then floor."""
    xmin, xmax, ymin, ymax = extent
    hx, hy = (xmax - xmin) / n, (ymax - ymin) / n
    det = np.stack([(det_xy[:, 0] - xmin) / hx - 0.5, (det_xy[:, 1] - ymin) / hy - 0.5], 1).astype(np.float32)
    phi = 2 * math.pi * (np.arange(quad_m) + 0.5) / quad_m
    cs = np.stack([np.cos(phi) / hx, np.sin(phi) / hy], 1).astype(np.float32)
    k = np.arange(n_t, dtype=np.float64)
    rk = (k * np.float64(np.float32(dr)) + np.float64(np.float32(r0 + 0.5 * dr))).astype(np.float32)
    r = rk.astype(np.float64)[None, :, None]
    fx = (r * cs[:, 0].astype(np.float64)[None, None, :] + det[:, 0].astype(np.float64)[:, None, None]).astype(np.float32)
    fy = (r * cs[:, 1].astype(np.float64)[None, None, :] + det[:, 1].astype(np.float64)[:, None, None]).astype(np.float32)
    return np.floor(fx).astype(np.int64), np.floor(fy).astype(np.int64)


def _window_member(win, M):
    """Boolean (units, M): angle m inside the window m_first | count << 16 (circular)."""
    first = (win & 0xFFFF).astype(np.int64)
    cnt = (win >> 16).astype(np.int64)
    m = np.arange(M)[None, :]
    return ((m - first[:, None]) % M) < cnt[:, None]


ROUND = 256


def _check_plan(n, det_xy, n_t, r0, dr, quad_m, sms, budget=0, extent=(-1.0, 1.0, -1.0, 1.0)):
    plan = P.pat_forward_plan(n, det_xy, n_t, r0, dr, quad_m, sms, budget, extent)
    units, ctas, roff, rgs = (plan[k].astype(np.int64) for k in ("units", "ctas", "roff", "rgs"))
    D, T, M = det_xy.shape[0], n_t, quad_m
    n_kgrp = (T + KGRP - 1) // KGRP
    S, R, W = plan["slabs"], plan["rows"], plan["stride"]
    assert 1 <= S <= 16
    if R > 0:
        assert S * R >= n + 1 and (S - 1) * R < n + 1            # the slabs cover j0 in [-1, N-1]
        if budget:
            assert (R + 1) * W * 4 <= budget
    else:
        assert S == 1
    assert W % 8 == 4 and W >= n + 6
    assert plan["smem"] <= 220 * 1024
    C = len(ctas)
    assert C % S == 0 and C >= S
    # every row group belongs to exactly one cluster
    assert np.array_equal(np.sort(rgs), np.arange(D * n_kgrp))
    unit_of = {}
    for c in range(C // S):
        g0, ng = ctas[c * S, 0], ctas[c * S, 1]
        assert np.all(ctas[c * S:(c + 1) * S, 0] == g0) and np.all(ctas[c * S:(c + 1) * S, 1] == ng) and ng >= 1
        n_rounds = (ng + ROUND - 1) // ROUND
        for rank in range(S):
            o = ctas[c * S + rank, 2]
            off = roff[o:o + n_rounds + 1]
            assert np.all(np.diff(off) >= 0)
            for rd in range(n_rounds):
                for u in range(off[rd], off[rd + 1]):
                    d, w0, w1, w = units[u]
                    kg, idx = w >> 16, w & 0xFFFF
                    assert 0 <= idx < min(ROUND, ng - rd * ROUND)
                    rg = rgs[g0 + rd * ROUND + idx]
                    assert rg == d * n_kgrp + kg, "unit names a row group outside its round"
                    assert (rg, rank) not in unit_of, "two units of one row group in one slab"
                    unit_of[(rg, rank)] = u
    assert sorted(set(range(len(units)))) == sorted(unit_of.values())
    # the two windows of a unit are disjoint
    w0 = _window_member(units[:, 1], M)
    w1 = _window_member(units[:, 2], M)
    assert not np.any(w0 & w1)
    cover = w0 | w1
    # brute force: every on-grid point is inside the windows of its (row group, slab) unit
    i0, j0 = _f32_points(n, det_xy, n_t, r0, dr, quad_m, extent)
    on = (i0 >= -1) & (i0 <= n - 1) & (j0 >= -1) & (j0 <= n - 1)
    d_idx, k_idx, m_idx = np.nonzero(on)
    s_pt = (j0[d_idx, k_idx, m_idx] + 1) // R if R > 0 else np.zeros_like(d_idx)
    rg_pt = d_idx * n_kgrp + k_idx // KGRP
    lut = -np.ones(D * n_kgrp * S, dtype=np.int64)
    for (rg, rank), u in unit_of.items():
        lut[rg * S + rank] = u
    u_pt = lut[rg_pt * S + s_pt]
    assert np.all(u_pt >= 0), "an on-grid point has no unit for its row group and slab"
    assert np.all(cover[u_pt, m_idx]), "an on-grid point lies outside its unit's windows"
    # the evaluated count is the windows' points over the valid radii of each unit
    nk = np.minimum(T - (units[:, 3] >> 16) * KGRP, KGRP)
    assert plan["evaluated"] == int(np.sum(cover.sum(1) * nk))
    assert plan["evaluated"] >= on.sum()
    return plan, int(on.sum())


GEOMS = {
    "full_circle": (24, S.detectors_full_circle(12, 1.2), 40, 0.0, 2.62 / 40, 64, (-1.0, 1.0, -1.0, 1.0)),
    "ragged_odd": (33, S.detectors_full_circle(7, 1.3), 45, 0.0, 2.8 / 45, 50, (-1.0, 1.0, -1.0, 1.0)),
    "limited_arc": (32, S.detectors_limited_arc(128, 32, 90.0, 5, 1.2), 70, 0.0, 2.7 / 70, 96, (-1.0, 1.0, -1.0, 1.0)),
    "centre_det": (20, np.array([[0.03, -0.05], [0.5, 0.4]]), 33, 0.0, 0.05, 200, (-1.0, 1.0, -1.0, 1.0)),
    "far_outside": (12, np.array([[4.0, 4.0]]), 8, 0.0, 0.2, 32, (-1.0, 1.0, -1.0, 1.0)),
    "non_square": (20, np.array([[2.0, 0.0], [0.0, 2.5], [-1.5, -1.0]]), 50, 0.2, 0.08, 80, (-1.5, 1.0, -0.5, 1.5)),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
@pytest.mark.parametrize("budget", [0, 2000, 400])
def test_forward_plan_small(name, budget):
    """Small geometries, with the library's budget (one slab here) and budgets small enough
    to force several slabs (2000 bytes) or the global-memory variant (400 bytes)."""
    n, det, n_t, r0, dr, m, ext = GEOMS[name]
    plan, on = _check_plan(n, det, n_t, r0, dr, m, sms=4, budget=budget, extent=ext)
    if budget == 400:
        assert plan["rows"] == 0
    if budget == 2000 and n >= 20:
        assert plan["slabs"] > 1


def test_forward_plan_benchmark_geometry():
    """The 256^2, 256 detectors x 512 samples, M = 256 workload with the library's budget."""
    w = S.workload("tgv256")
    plan, on = _check_plan(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"], sms=152)
    assert plan["slabs"] >= 2 and plan["rows"] >= 8
    assert plan["evaluated"] <= 1.2 * on          # the windows add little beyond the grid's points
    assert len(plan["ctas"]) >= 200
    # the CTAs' work is balanced: the largest is close to the mean
    cnt = (plan["units"][:, 1] >> 16) + (plan["units"][:, 2] >> 16)
    ctas, roff = plan["ctas"], plan["roff"]
    work = np.array([cnt[roff[o]:roff[o + 1 + (ng + 255) // 256 - 1]].sum() for _, ng, o, _ in ctas])
    assert work.max() <= 1.15 * work.mean()


def test_forward_plan_limited_angle_geometry():
    w = S.workload("dtv256")
    _check_plan(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"], sms=152)
