"""Host logic of the K^T work list (pat_adjoint_worklist; no GPU needed).

The K^T kernel adds, for every pixel tile, the candidate points that the host's ray
segments list, and it tests each candidate's taps exactly.  So the list must hold every
point that has a tap in the tile (else a term of K^T y is lost), and the work items must
cut each tile's list into disjoint pieces that cover it (else a term is lost or counted
twice).  Both are checked here by brute force over every quadrature point
(d, k, m) of Sec. 4.2's discretisation, with the FP32 point arithmetic of the kernels.
A mirror of the kernel's traversal (per-thread runs, the binary search for a run's first
segment, the segment switches) checks that every candidate of an item is visited once.
"""
import math

import numpy as np
import pytest

import paper_1707_02245_gb300 as P
import synthetic as S

WTILE = 32   # side of the K^T work tiles
ARAYS = 1024


def _tables(n, det_xy, n_t, r0, dr, quad_m, extent=(-1.0, 1.0, -1.0, 1.0)):
    """FP32 detector positions and (cos, sin) in pixel units and radii, as the device holds them."""
    xmin, xmax, ymin, ymax = extent
    hx, hy = (xmax - xmin) / n, (ymax - ymin) / n
    det = np.stack([(det_xy[:, 0] - xmin) / hx - 0.5, (det_xy[:, 1] - ymin) / hy - 0.5], 1).astype(np.float32)
    phi = 2 * math.pi * (np.arange(quad_m) + 0.5) / quad_m
    cs = np.stack([np.cos(phi) / hx, np.sin(phi) / hy], 1).astype(np.float32)
    # r_k = fmaf(k, dr, r0 + dr/2) in FP32: the exact product plus the constant, rounded once
    k = np.arange(n_t, dtype=np.float64)
    rk = (k * np.float64(np.float32(dr)) + np.float64(np.float32(r0 + 0.5 * dr))).astype(np.float32)
    return det, cs, rk


def _check_worklist(n, det_xy, n_t, r0, dr, quad_m, slots, extent=(-1.0, 1.0, -1.0, 1.0)):
    wl = P.pat_adjoint_worklist(n, det_xy, n_t, r0, dr, quad_m, slots, extent)
    rays, items = wl["rays"], wl["items"]
    D, T, M = det_xy.shape[0], n_t, quad_m
    tiles_x = (n + WTILE - 1) // WTILE
    tiles = tiles_x * tiles_x

    # per tile: segments with increasing prefixes, then a sentinel with the total
    sent = np.flatnonzero(rays[:, 0] == -1)
    assert sent.size == tiles
    k0 = np.zeros((tiles, D, M), dtype=np.int64)
    k1 = np.zeros((tiles, D, M), dtype=np.int64)
    base, total = 0, 0
    tile_total = np.zeros(tiles, dtype=np.int64)
    for t in range(tiles):
        seg = rays[base:sent[t]]
        pre = np.append(seg[:, 3], rays[sent[t], 3])
        assert pre[0] == 0 and np.all(np.diff(pre) > 0), f"tile {t}: empty or unordered segment"
        assert np.all((seg[:, 0] >= 0) & (seg[:, 0] < D) & (seg[:, 1] >= 0) & (seg[:, 1] < M))
        ln = np.diff(pre)
        assert np.all(seg[:, 2] >= 0) and np.all(seg[:, 2] + ln <= T)
        # one segment per (detector, angle) in a tile
        assert np.unique(seg[:, 0].astype(np.int64) * M + seg[:, 1]).size == seg.shape[0]
        k0[t, seg[:, 0], seg[:, 1]] = seg[:, 2]
        k1[t, seg[:, 0], seg[:, 1]] = seg[:, 2] + ln
        tile_total[t] = pre[-1]
        total += pre[-1]
        base = sent[t] + 1
    assert base == rays.shape[0]
    assert wl["candidates"] == total

    # items: disjoint pieces covering each tile's list, with consistent segment ranges
    covered = {t: [] for t in range(tiles)}
    for tile, ray0, nray, c0, c1 in items:
        if nray == 0:
            assert c0 == c1 == 0 and total == 0
            continue
        assert 1 <= nray <= ARAYS and c0 < c1
        assert rays[ray0, 0] >= 0 and rays[ray0 + nray - 1, 0] >= 0
        assert rays[ray0, 3] <= c0 < rays[ray0 + 1, 3], "first segment does not hold c0"
        assert rays[ray0 + nray - 1, 3] < c1 <= rays[ray0 + nray, 3], "last segment does not hold c1 - 1"
        # all of the item's segments belong to its tile
        t_first = 0 if tile == 0 else sent[tile - 1] + 1
        assert t_first <= ray0 and ray0 + nray <= sent[tile]
        covered[tile].append((c0, c1))
    for t in range(tiles):
        iv = sorted(covered[t])
        if tile_total[t] == 0:
            assert not iv
            continue
        assert iv[0][0] == 0 and iv[-1][1] == tile_total[t]
        assert all(a[1] == b[0] for a, b in zip(iv, iv[1:])), f"tile {t}: pieces overlap or leave a gap"

    # every point with a tap in a tile is a candidate of that tile (FP32 point arithmetic)
    det, cs, rk = _tables(n, det_xy, n_t, r0, dr, quad_m, extent)
    dd, kk, mm = np.meshgrid(np.arange(D), np.arange(T), np.arange(M), indexing="ij")
    dd, kk, mm = dd.ravel(), kk.ravel(), mm.ravel()
    fx = (rk[kk].astype(np.float64) * cs[mm, 0] + det[dd, 0]).astype(np.float32)
    fy = (rk[kk].astype(np.float64) * cs[mm, 1] + det[dd, 1]).astype(np.float32)
    i0 = np.floor(fx).astype(np.int64)
    j0 = np.floor(fy).astype(np.int64)
    missing = 0
    for di in (0, 1):
        for dj in (0, 1):
            ti, tj = i0 + di, j0 + dj
            on = (ti >= 0) & (ti < n) & (tj >= 0) & (tj < n)
            tile = (tj[on] // WTILE) * tiles_x + ti[on] // WTILE
            d_, k_, m_ = dd[on], kk[on], mm[on]
            ok = (k0[tile, d_, m_] <= k_) & (k_ < k1[tile, d_, m_])
            missing += int(np.count_nonzero(~ok))
    assert missing == 0, f"{missing} (point, tap) pairs have no candidate in their tile"
    return wl


def _full_circle(n_det, radius):
    a = 2 * math.pi * (np.arange(n_det) + 0.5) / n_det
    return np.stack([radius * np.cos(a), radius * np.sin(a)], 1)


@pytest.mark.parametrize("name", ["small", "disc64"])
def test_worklist_covers_every_point_of_the_test_workloads(name):
    w = S.workload(name)
    _check_worklist(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"], slots=4 * 152)


def test_worklist_limited_arc_and_ragged_tiles():
    # 90 degree arc, N not a multiple of the tile side (ragged last tile row and column)
    det = S.detectors_limited_arc(128, 24, 90.0, 5, radius=1.2)
    r0, dr = S.radial_sampling(det, 96)
    _check_worklist(72, det, 96, r0, dr, 128, slots=608)


def test_worklist_detectors_inside_the_image():
    # detectors inside the square: boxes of the tiles around them span every angle
    det = _full_circle(16, 0.55)
    r0, dr = S.radial_sampling(det, 80)
    _check_worklist(40, det, 80, r0, dr, 96, slots=64)


def test_worklist_non_square_extent():
    # rectangular pixels (h_x != h_y) and detectors off-centre on both sides
    det = np.array([[2.0, 0.0], [0.0, 2.5], [-1.5, -1.0], [0.3, 1.2]])
    extent = (-1.5, 1.0, -0.5, 1.5)
    far = max(math.hypot(dx - cx, dy - cy) for dx, dy in det for cx in extent[:2] for cy in extent[2:])
    n_t = 90
    _check_worklist(40, det, n_t, 0.1, far / n_t, 112, slots=24, extent=extent)


def test_worklist_pieces_fill_one_wave():
    # at the benchmark's geometry the items are exactly one wave of resident CTAs, of
    # nearly equal size (no partial wave)
    w = S.workload("tgv256")
    for slots in (5 * 152, 6 * 152):
        wl = P.pat_adjoint_worklist(w["n"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"], slots)
        it = wl["items"]
        sizes = it[:, 4] - it[:, 3]
        assert it.shape[0] == slots
        assert sizes.max() <= 1.15 * wl["candidates"] / slots
        assert sizes.sum() == wl["candidates"]


def test_worklist_rejects_bad_input():
    with pytest.raises(P.PatError):
        P.pat_adjoint_worklist(1, np.zeros((1, 2)), 10, 0.0, 0.1, 16, slots=8)


ATHREADS = 256   # threads of a K^T CTA


def _pow2_at_least(x):
    return 1 if x <= 1 else 2 * _pow2_at_least((x + 1) // 2)


def _kernel_visits(rays, item):
    """The (segment, k) pairs the K^T kernel's threads visit for one work item: thread t
    takes the run [c0 + tC, c0 + (t+1)C), finds its first segment by the kernel's binary
    search (halving steps from the power of two ASTEP), then walks the run in one loop that
    moves to the next segment when the run crosses a segment end."""
    tile, ray0, nray, c0, c1 = (int(v) for v in item)
    s_ray = rays[ray0:ray0 + nray + 1]
    astep = _pow2_at_least(ARAYS) // 2
    C = (c1 - c0 + ATHREADS - 1) // ATHREADS
    out = []
    for t in range(ATHREADS):
        p = c0 + t * C
        p_end = min(c1, p + C)
        if p >= p_end:
            continue
        j, step = 0, astep
        while step > 0:
            if j + step < nray and s_ray[j + step, 3] <= p:
                j += step
            step >>= 1
        seg_end = int(s_ray[j + 1, 3])
        k = int(s_ray[j, 2]) + (p - int(s_ray[j, 3]))
        while p < p_end:
            if p == seg_end:
                j += 1
                assert j < nray, "run left the item's segments"
                seg_end = int(s_ray[j + 1, 3])
                k = int(s_ray[j, 2])
            out.append((ray0 + j, k))
            p += 1
            k += 1
    return out


@pytest.mark.parametrize("slots", [3, 40, 608])
def test_kernel_traversal_visits_each_candidate_once(slots):
    # the candidates of every item, visited as the kernel's threads do, are exactly the
    # item's slice of its tile's list; over all items every candidate appears once
    det = S.detectors_limited_arc(128, 24, 90.0, 5, radius=1.2)
    r0, dr = S.radial_sampling(det, 96)
    wl = P.pat_adjoint_worklist(72, det, 96, r0, dr, 128, slots)
    rays, items = wl["rays"], wl["items"]
    seen = []
    for it in items:
        tile, ray0, nray, c0, c1 = (int(v) for v in it)
        if nray == 0:
            continue
        got = _kernel_visits(rays, it)
        # expected: walk the tile's segments from the one holding c0
        exp = []
        j = ray0
        for c in range(c0, c1):
            while rays[j + 1, 3] <= c:
                j += 1
            exp.append((j, int(rays[j, 2]) + c - int(rays[j, 3])))
        assert got == exp
        seen += got
    assert len(seen) == len(set(seen)) == wl["candidates"]


def test_kernel_traversal_binary_search_many_segments():
    # items with hundreds of segments (short rays near a detector inside the image) reach
    # deep into the binary search; each run must start on the segment that holds it
    det = _full_circle(16, 0.55)
    r0, dr = S.radial_sampling(det, 80)
    wl = P.pat_adjoint_worklist(40, det, 80, r0, dr, 96, slots=2)
    items = wl["items"]
    assert items[:, 2].max() > 64
    total = 0
    for it in items:
        total += len(_kernel_visits(wl["rays"], it))
    assert total == wl["candidates"]
