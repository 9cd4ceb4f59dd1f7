"""Plain FP64 CPU oracle for the measurement pre-processing of Sec. 4.3 (before the
reconstruction: the data f of min 1/2 ||Ku - f||^2 + alpha R(u) are made from measured
pressures p).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module.  The CUDA library never imports,
links or executes it, and it shares no code, tables or helpers with the CUDA path.

What it computes, per detector d at x_d, for a calibration pulse source at x_p:
1. The regularised deconvolution (eq. (deconv)):
     f_t = F^-1{ F{p} conj(F{h}) / (|F{h}|^2 + eps) },
   where h is the calibration measurement p_cal moved to the retarded time
   t' = t - |x_d - x_p| / c0 (eq. (FW_full)).
2. The rescale (eq. (f_rewrite)): f = t / |x_d - x_p| * f_t.

Readings where the paper is silent:
P1  Sampling.  Samples sit at t_k = r0 + (k + 1/2) dr (speed of sound c0 = 1, so
    time = radius, as for K).  The time convolution of eq. (FW_conv) is discretised as
    dr * sum_m f_t[k - m] h[m].
P2  Transform length.  The DFT has length L = the smallest power of two >= 2T, with the
    zero-padded signals, so that the product in the frequency domain stands for a linear
    (not wrapped) convolution of two T-sample signals.  The first T samples of the inverse
    are kept.
P3  Retarded time.  h[m] = p_cal(m dr + |x_d - x_p|), the calibration advanced by the
    travel time.  It is formed from the samples of p_cal by the exact shift theorem for
    band-limited signals: the DFT is multiplied by exp(+2 pi i nu delta / L) with the
    signed frequency index nu in [-L/2, L/2) and delta = (|x_d - x_p| - t_0) / dr
    samples.  At nu = -L/2 the cosine of the phase is kept, so a real signal stays real.
P4  eps.  It is given relative to the largest |F{h}|^2 of the detector:
    eps = eps_rel * max_nu |F{h}(nu)|^2.

Pins (tests/test_prep_oracle_pins.py):
- the deconvolution equals the Tikhonov minimiser of |C f - p|^2 + eps |f|^2 for the
  circulant C of dr h, from a dense solve;
- an integer delay equals np.roll;
- a unit-impulse calibration with eps -> 0 returns p, advanced by the delay and rescaled;
- the rescale is a closed form.
"""
from __future__ import annotations

import math

import numpy as np


def transform_length(n_t: int) -> int:
    """Reading P2: the smallest power of two >= 2 T."""
    L = 1
    while L < 2 * n_t:
        L *= 2
    return L


def signed_freqs(L: int) -> np.ndarray:
    """Signed DFT frequency indices nu in [-L/2, L/2), in the DFT's order."""
    return np.fft.fftfreq(L, d=1.0 / L)


def shift_spectrum(H: np.ndarray, delta: float) -> np.ndarray:
    """Spectrum of the signal advanced by ``delta`` samples (reading P3): multiply by
    exp(+2 pi i nu delta / L); at the Nyquist index only the cosine is kept."""
    L = H.shape[-1]
    nu = signed_freqs(L)
    ph = np.exp(2j * math.pi * nu * delta / L)
    ph[L // 2] = math.cos(math.pi * delta)    # nu = -L/2: real part of the phase
    return H * ph


def calibration_kernel_spectrum(p_cal_d: np.ndarray, dist: float, t0: float, dr: float, L: int) -> np.ndarray:
    """F{dr h} of one detector: the zero-padded calibration, advanced by its travel time
    (readings P1, P3)."""
    P = np.fft.fft(np.concatenate([np.asarray(p_cal_d, dtype=np.float64), np.zeros(L - len(p_cal_d))]))
    return dr * shift_spectrum(P, (dist - t0) / dr)


def deconvolve_detector(p_d, p_cal_d, dist: float, t0: float, dr: float, eps_rel: float) -> np.ndarray:
    """f_t of one detector (eq. (deconv) with readings P1-P4); returns T samples."""
    T = len(p_d)
    L = transform_length(T)
    H = calibration_kernel_spectrum(p_cal_d, dist, t0, dr, L)
    Pp = np.fft.fft(np.concatenate([np.asarray(p_d, dtype=np.float64), np.zeros(L - T)]))
    eps = eps_rel * float(np.max(np.abs(H) ** 2))
    F = Pp * np.conj(H) / (np.abs(H) ** 2 + eps)
    return np.real(np.fft.ifft(F))[:T]


def preprocess(p, p_cal, det_xy, xp, r0: float, dr: float, eps_rel: float) -> np.ndarray:
    """Pre-processed data f (D x T) from pressures p and calibrations p_cal (D x T):
    deconvolution, then f = t / |x_d - x_p| f_t (eq. (f_rewrite))."""
    p = np.asarray(p, dtype=np.float64)
    D, T = p.shape
    t = r0 + (np.arange(T) + 0.5) * dr
    out = np.zeros((D, T))
    for d in range(D):
        dist = math.hypot(det_xy[d][0] - xp[0], det_xy[d][1] - xp[1])
        ft = deconvolve_detector(p[d], p_cal[d], dist, t[0], dr, eps_rel)
        out[d] = t / dist * ft
    return out
