"""Seeded synthetic inputs for photoacoustic reconstruction workloads.

This module only draws random numbers and rasterises shapes: detector layouts,
phantom images, side images for directional TV, and standard-normal noise
arrays.  It contains none of the reconstruction method's arithmetic (no
projector, no finite differences, no prox maps, no step sizes), so both the CPU
oracle and the CUDA path can be fed from it without sharing method code.

The workloads stand in for the paper's test objects (Sec. 5.1): piecewise
constant discs for the TV experiments, a smooth decaying fluence for TGV, and a
vascular structure.  The paper's vascular phantom came from a retinal image
database that is not available here; a seeded random vessel tree of line
segments replaces it.  All images live on the square [-1, 1]^2 with row-major
layout ``img[iy, ix]`` and pixel centres at ``-1 + (i + 1/2) * 2/N``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Disc",
    "detectors_full_circle",
    "detectors_limited_arc",
    "disc_params",
    "rasterise_discs",
    "disc_phantom",
    "vessel_segments",
    "rasterise_segments",
    "vessel_phantom",
    "side_image",
    "standard_normal",
    "uniform",
    "pixel_centres",
    "radial_sampling",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def pixel_centres(n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Coordinates of the n pixel centres along one axis of [lo, hi]."""
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


# ----------------------------------------------------------------------------
# detector layouts (point detectors in the image plane, Sec. 3.3.1)
# ----------------------------------------------------------------------------

def detectors_full_circle(n_det: int, radius: float = 1.2) -> np.ndarray:
    """``n_det`` point detectors evenly spaced on a full circle; shape (n_det, 2)."""
    ang = 2.0 * math.pi * np.arange(n_det, dtype=np.float64) / n_det
    return np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1)


def detectors_limited_arc(n_total: int, n_keep: int, arc_deg: float, seed: int,
                          radius: float = 1.2, centre_deg: float = 0.0) -> np.ndarray:
    """Compressive limited-angle layout.

    ``n_total`` positions spaced evenly over an arc of ``arc_deg`` degrees centred
    at ``centre_deg``; ``n_keep`` of them are drawn without replacement from the
    seed and returned in angular order; shape (n_keep, 2).
    """
    half = math.radians(arc_deg) / 2.0
    c = math.radians(centre_deg)
    if n_total == 1:
        ang = np.array([c])
    else:
        ang = c - half + 2.0 * half * np.arange(n_total, dtype=np.float64) / (n_total - 1)
    keep = np.sort(_rng(seed).choice(n_total, size=n_keep, replace=False))
    ang = ang[keep]
    return np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1)


# ----------------------------------------------------------------------------
# disc phantoms (piecewise constant, Sec. 5.1 first phantom)
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Disc:
    cx: float
    cy: float
    radius: float
    amplitude: float


def disc_params(n_discs: int, seed: int, r_lo: float = 0.05, r_hi: float = 0.2,
                a_lo: float = 0.5, a_hi: float = 1.0, support: float = 1.0) -> list[Disc]:
    """Random uniform discs: radius U[r_lo, r_hi], amplitude U[a_lo, a_hi].

    Centres are uniform in the disc |c| <= support - radius, so every disc lies
    inside the unit circle.
    """
    g = _rng(seed)
    out = []
    for _ in range(n_discs):
        rad = g.uniform(r_lo, r_hi)
        amp = g.uniform(a_lo, a_hi)
        rho = (support - rad) * math.sqrt(g.uniform(0.0, 1.0))
        phi = g.uniform(0.0, 2.0 * math.pi)
        out.append(Disc(rho * math.cos(phi), rho * math.sin(phi), rad, amp))
    return out


def rasterise_discs(discs: list[Disc], n: int, supersample: int = 4) -> np.ndarray:
    """Sum of disc indicators, averaged over ``supersample``^2 sub-pixel samples."""
    h = 2.0 / n
    sub = (np.arange(supersample, dtype=np.float64) + 0.5) / supersample
    xs = (-1.0 + (np.arange(n)[:, None] + sub[None, :]) * h).reshape(-1)
    X, Y = np.meshgrid(xs, xs)  # (n*ss, n*ss), Y varies along rows
    img = np.zeros_like(X)
    for dsc in discs:
        img += dsc.amplitude * (((X - dsc.cx) ** 2 + (Y - dsc.cy) ** 2) <= dsc.radius ** 2)
    return img.reshape(n, supersample, n, supersample).mean(axis=(1, 3))


def disc_phantom(n: int, n_discs: int, seed: int, supersample: int = 4) -> tuple[np.ndarray, list[Disc]]:
    discs = disc_params(n_discs, seed)
    return rasterise_discs(discs, n, supersample), discs


# ----------------------------------------------------------------------------
# vessel tree (stand-in for the retinal vascular phantom, Sec. 5.1)
# ----------------------------------------------------------------------------

def vessel_segments(seed: int, n_segments: int = 40, n_pix: int = 256,
                    w_lo_px: float = 1.0, w_hi_px: float = 4.0,
                    support: float = 0.95) -> np.ndarray:
    """A random branching tree of line segments.

    Returns an array (n_segments, 5): x0, y0, x1, y1, width (in image units).
    The tree grows from a root near the unit circle towards the centre; each new
    segment starts at the end point of a random earlier segment, turns by a
    random angle and is thinner than its parent.  Widths are drawn in pixel
    units of an ``n_pix`` grid so that they stay 1-4 pixels wide.
    """
    g = _rng(seed)
    h = 2.0 / n_pix
    segs = []
    ang0 = g.uniform(0.0, 2.0 * math.pi)
    start = np.array([support * math.cos(ang0), support * math.sin(ang0)])
    heading = ang0 + math.pi + g.uniform(-0.3, 0.3)
    widths = []
    ends = []
    headings = []
    w = w_hi_px
    for s in range(n_segments):
        if s > 0:
            parent = int(g.integers(0, len(segs)))
            start = ends[parent]
            heading = headings[parent] + g.choice([-1.0, 1.0]) * g.uniform(0.25, 0.9)
            w = max(w_lo_px, widths[parent] * g.uniform(0.65, 0.95))
        length = g.uniform(0.15, 0.45)
        end = start + length * np.array([math.cos(heading), math.sin(heading)])
        rad = float(np.hypot(*end))
        if rad > support:  # pull the end point back inside the support
            end = end * (support / rad)
        segs.append([start[0], start[1], end[0], end[1], w * h])
        widths.append(w)
        ends.append(end)
        headings.append(heading)
    return np.asarray(segs, dtype=np.float64)


def rasterise_segments(segs: np.ndarray, n: int, supersample: int = 4) -> np.ndarray:
    """Union of thick segments (capsules) averaged over sub-pixel samples; values in [0, 1]."""
    h = 2.0 / n
    m = n * supersample
    sub_h = h / supersample
    coords = -1.0 + (np.arange(m, dtype=np.float64) + 0.5) * sub_h
    mask = np.zeros((m, m), dtype=bool)
    for x0, y0, x1, y1, w in segs:
        half = 0.5 * w
        lo_x = max(0, int((min(x0, x1) - half + 1.0) / sub_h) - 1)
        hi_x = min(m, int((max(x0, x1) + half + 1.0) / sub_h) + 2)
        lo_y = max(0, int((min(y0, y1) - half + 1.0) / sub_h) - 1)
        hi_y = min(m, int((max(y0, y1) + half + 1.0) / sub_h) + 2)
        if lo_x >= hi_x or lo_y >= hi_y:
            continue
        X, Y = np.meshgrid(coords[lo_x:hi_x], coords[lo_y:hi_y])
        dx, dy = x1 - x0, y1 - y0
        ll = dx * dx + dy * dy
        t = np.clip(((X - x0) * dx + (Y - y0) * dy) / ll, 0.0, 1.0) if ll > 0 else np.zeros_like(X)
        dist2 = (X - x0 - t * dx) ** 2 + (Y - y0 - t * dy) ** 2
        mask[lo_y:hi_y, lo_x:hi_x] |= dist2 <= half * half
    return mask.reshape(n, supersample, n, supersample).mean(axis=(1, 3))


def vessel_phantom(n: int, seed: int, n_segments: int = 40, mu: float = 3.0,
                   supersample: int = 4, n_ref: int | None = None) -> np.ndarray:
    """Vessel tree times an exponentially decaying fluence exp(-mu * depth).

    depth = max(0, 1 - |x|) is the distance inward from the unit circle, so the
    absorbed energy is largest near the illuminated boundary.  Vessel widths are
    1-4 pixels of an ``n_ref`` grid (default ``n``), so the same tree can be
    rasterised on a finer grid.
    """
    segs = vessel_segments(seed, n_segments=n_segments, n_pix=n_ref or n)
    mask = rasterise_segments(segs, n, supersample)
    c = pixel_centres(n)
    X, Y = np.meshgrid(c, c)
    depth = np.maximum(0.0, 1.0 - np.hypot(X, Y))
    return mask * np.exp(-mu * depth)


def side_image(n: int, seed: int, n_segments: int = 40, blur_px: float = 1.5,
               background: float = 0.2) -> np.ndarray:
    """Side image for directional TV sharing the vessel edges of ``vessel_phantom``.

    The vessel mask of the same seed is smoothed with a separable Gaussian of
    ``blur_px`` pixels and a smooth seeded background (a few low-frequency
    cosines) is added.
    """
    segs = vessel_segments(seed, n_segments=n_segments, n_pix=n)
    mask = rasterise_segments(segs, n, 4)
    rad = max(1, int(math.ceil(3 * blur_px)))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (t / blur_px) ** 2)
    ker /= ker.sum()
    pad = np.pad(mask, rad, mode="edge")
    tmp = np.apply_along_axis(lambda v: np.convolve(v, ker, mode="valid"), 1, pad)
    sm = np.apply_along_axis(lambda v: np.convolve(v, ker, mode="valid"), 0, tmp)
    g = _rng(seed + 7919)
    c = pixel_centres(n)
    X, Y = np.meshgrid(c, c)
    bg = np.zeros_like(X)
    for _ in range(3):
        kx, ky = g.uniform(0.3, 1.5, size=2)
        ph = g.uniform(0.0, 2.0 * math.pi)
        bg += np.cos(math.pi * (kx * X + ky * Y) + ph)
    return sm + background * bg / 3.0


# ----------------------------------------------------------------------------
# noise
# ----------------------------------------------------------------------------

def standard_normal(shape, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal(shape)


def uniform(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return _rng(seed).uniform(lo, hi, size=shape)


def radial_sampling(det_xy: np.ndarray, n_t: int, lo: float = -1.0, hi: float = 1.0) -> tuple[float, float]:
    """(r0, dr) so that the radii r_k = r0 + (k + 1/2) dr, k < n_t, cover the square.

    r0 = 0 and dr = r_max / n_t with r_max the largest detector-to-corner distance
    (speed of sound 1, so time samples are radii).
    """
    det = np.asarray(det_xy, dtype=np.float64).reshape(-1, 2)
    corners = np.array([[lo, lo], [lo, hi], [hi, lo], [hi, hi]])
    rmax = float(np.max(np.hypot(det[:, None, 0] - corners[None, :, 0],
                                 det[:, None, 1] - corners[None, :, 1])))
    return 0.0, rmax / n_t


# ----------------------------------------------------------------------------
# workload recipes (sizes, layouts, phantoms, noise draws; no operator applied)
# ----------------------------------------------------------------------------

def workload(name: str, seed: int = 0) -> dict:
    """Inputs of a named reconstruction workload.

    Keys: n, det_xy, n_t, r0, dr, quad_m (reconstruction grid), n_fine, quad_m_fine
    and phantom_fine (data are simulated on a 2x finer grid with 2x the quadrature so
    the reconstruction does not commit an inverse crime, Sec. 5.2), phantom (at n),
    noise (standard normal, shape (D, T)), noise_level (std as a fraction of the clean
    data's maximum), reg / alpha / beta / gamma / iters, and for directional TV the
    side image ``side`` and ``eta``.

    * ``disc64``:   64^2 image, 64 detectors on a full circle of radius 1.2, 128 time
      samples, 256 quadrature points, 5 random discs, 1% noise, TV alpha 0.05, 200 its.
    * ``tgv256``:   256^2 vessel tree with exp(-3 depth) fluence, 256 detectors on the
      full circle, 512 samples, 5% noise, TGV alpha 0.02 beta 0.04, 1000 iterations.
    * ``dtv256``:   the tgv256 phantom, 32 of 128 detectors on a 90 degree arc, 512
      samples, 10% noise, directional TV alpha 0.02, gamma 0.95, 2000 iterations.
    * ``small``:    a few-second case for tests: 24^2 discs, 12 detectors, 40 samples,
      64 quadrature points, 2% noise.
    """
    if name == "disc64":
        n, n_det, n_t, m = 64, 64, 128, 256
        det = detectors_full_circle(n_det, 1.2)
        discs = disc_params(5, seed)
        ph = rasterise_discs(discs, n)
        ph_f = rasterise_discs(discs, 2 * n)
        out = dict(reg=0, alpha=0.05, beta=1.0, gamma=0.95, iters=200, noise_level=0.01)
    elif name == "small":
        n, n_det, n_t, m = 24, 12, 40, 64
        det = detectors_full_circle(n_det, 1.2)
        discs = disc_params(3, seed)
        ph = rasterise_discs(discs, n)
        ph_f = rasterise_discs(discs, 2 * n)
        out = dict(reg=0, alpha=0.05, beta=1.0, gamma=0.95, iters=50, noise_level=0.02)
    elif name in ("tgv256", "dtv256"):
        n, n_t, m = 256, 512, 256
        if name == "tgv256":
            det = detectors_full_circle(256, 1.2)
            out = dict(reg=1, alpha=0.02, beta=0.04, gamma=0.95, iters=1000, noise_level=0.05)
        else:
            det = detectors_limited_arc(128, 32, 90.0, seed + 101, radius=1.2)
            out = dict(reg=2, alpha=0.02, beta=1.0, gamma=0.95, iters=2000, noise_level=0.10)
        ph = vessel_phantom(n, seed)
        ph_f = vessel_phantom(2 * n, seed, n_ref=n)
    else:
        raise ValueError(f"unknown workload {name!r}")
    r0, dr = radial_sampling(det, n_t)
    out.update(name=name, seed=seed, n=n, det_xy=det, n_t=n_t, r0=r0, dr=dr, quad_m=m,
               n_fine=2 * n, quad_m_fine=2 * m, phantom=ph, phantom_fine=ph_f,
               noise=standard_normal((det.shape[0], n_t), seed + 17))
    if out["reg"] == 2:
        w = side_image(n, seed)
        out["side"] = w
        out["eta"] = 0.01 * float(w.max() - w.min())
    return out


def workload_batch(seed: int = 0, count: int = 64) -> list[dict]:
    """A batch of uneven independent reconstructions (the mixed batched workload).

    Per problem: image side N from {128, 192, 256, 384, 512}, detector count from
    {32, 64, 128, 256, 512} on a full circle of radius 1.2, T = 2N time samples,
    M = 256; regulariser TV, TGV or directional TV in equal thirds; alpha log-uniform in
    [1e-3, 1e-1]; phantom a disc set or a vessel tree (alternating); noise level U[1%, 10%].
    Same keys as ``workload``.
    """
    g = _rng(seed + 4242)
    sizes = [128, 192, 256, 384, 512]
    dets = [32, 64, 128, 256, 512]
    out = []
    for i in range(count):
        n = int(g.choice(sizes))
        n_det = int(g.choice(dets))
        n_t = 2 * n
        reg = i % 3
        alpha = float(10.0 ** g.uniform(-3.0, -1.0))
        level = float(g.uniform(0.01, 0.10))
        pseed = int(g.integers(0, 2**31 - 1))
        det = detectors_full_circle(n_det, 1.2)
        if i % 2 == 0:
            discs = disc_params(5, pseed)
            ph, ph_f = rasterise_discs(discs, n, 2), rasterise_discs(discs, 2 * n, 2)
        else:
            ph = vessel_phantom(n, pseed, supersample=2)
            ph_f = vessel_phantom(2 * n, pseed, n_ref=n, supersample=2)
        r0, dr = radial_sampling(det, n_t)
        w = dict(name=f"batch{i}", seed=pseed, n=n, det_xy=det, n_t=n_t, r0=r0, dr=dr, quad_m=256,
                 n_fine=2 * n, quad_m_fine=512, phantom=ph, phantom_fine=ph_f,
                 noise=standard_normal((n_det, n_t), pseed + 17), noise_level=level,
                 reg=reg, alpha=alpha, beta=2.0 if reg == 1 else 1.0, gamma=0.95, iters=1000)
        if reg == 2:
            side = side_image(n, pseed) if i % 2 == 1 else rasterise_discs(disc_params(5, pseed), n)
            w["side"] = side
            w["eta"] = 0.01 * float(side.max() - side.min())
        out.append(w)
    return out


def workload_warm(seed: int, n: int = 256, n_det: int = 128, n_t: int | None = None, quad_m: int = 256) -> dict:
    """One problem of the learned-warm-start set: an n^2 vessel tree with exp(-3 depth)
    fluence, ``n_det`` detectors on a full circle of radius 1.2, T = 2n time samples by
    default, noise level U[1%, 10%] drawn from the seed, TGV alpha 0.02, beta 0.04.
    Same keys as ``workload``; seeds index the set (training and held-out seeds are
    disjoint ranges chosen by the caller)."""
    g = _rng(seed + 90001)
    level = float(g.uniform(0.01, 0.10))
    n_t = n_t or 2 * n
    det = detectors_full_circle(n_det, 1.2)
    r0, dr = radial_sampling(det, n_t)
    ph = vessel_phantom(n, seed, supersample=2, n_ref=max(n, 64))
    ph_f = vessel_phantom(2 * n, seed, n_ref=max(n, 64), supersample=2)
    return dict(name=f"warm{seed}", seed=seed, n=n, det_xy=det, n_t=n_t, r0=r0, dr=dr, quad_m=quad_m,
                n_fine=2 * n, quad_m_fine=2 * quad_m, phantom=ph, phantom_fine=ph_f,
                noise=standard_normal((n_det, n_t), seed + 17), noise_level=level,
                reg=1, alpha=0.02, beta=0.04, gamma=0.95, iters=1000)


def calibration_pulse(t, width: float, bipolar: bool = True):
    """Photoacoustic calibration pulse centred at c = 4 width (causal to within exp(-8)):
    bipolar, -(t - c) / width * exp(-(t - c)^2 / (2 width^2)) (the time derivative of a
    Gaussian illumination profile, detector response idealised), or the Gaussian itself."""
    t = np.asarray(t, dtype=np.float64)
    c = 4.0 * width
    g = np.exp(-0.5 * ((t - c) / width) ** 2)
    return -(t - c) / width * g if bipolar else g


def pressure_measurement(f, det_xy, xp, r0: float, dr: float, width: float, noise_level: float, seed: int,
                         bipolar: bool = True):
    """Synthetic pressures p and calibrations p_cal (D x T) for data f (D x T) on the samples
    t_k = r0 + (k + 1/2) dr, the measurement model of Sec. 4.3:
    p = (|x_d - x_p| / t f) * h with the pulse h(s) = calibration_pulse(s) (time convolution,
    dr * sum, linear and causal), and p_cal[d, k] = calibration_pulse(t_k - |x_d - x_p|),
    the calibration measured from the pulse source x_p.  Gaussian noise of std
    noise_level * max|.| is added to both."""
    f = np.asarray(f, dtype=np.float64)
    D, T = f.shape
    t = r0 + (np.arange(T) + 0.5) * dr
    dist = np.hypot(det_xy[:, 0] - xp[0], det_xy[:, 1] - xp[1])
    h = calibration_pulse(np.arange(T) * dr, width, bipolar)
    p = np.zeros((D, T))
    for d in range(D):
        ft = dist[d] / t * f[d]
        p[d] = dr * np.convolve(ft, h)[:T]
    pcal = calibration_pulse(t[None, :] - dist[:, None], width, bipolar)
    g = _rng(seed + 555)
    p += noise_level * np.abs(p).max() * g.standard_normal(p.shape)
    pcal += noise_level * np.abs(pcal).max() * g.standard_normal(pcal.shape)
    return p, pcal
