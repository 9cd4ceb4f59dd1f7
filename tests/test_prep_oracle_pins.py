"""Pins for the FP64 oracle of the measurement pre-processing (oracle/prep_oracle.py):

* the regularised deconvolution equals the Tikhonov minimiser of |C f - p|^2 + eps |f|^2
  for the circulant C of the kernel, solved densely (no FFT);
* the shift theorem with an integer delay equals np.roll;
* a unit-impulse calibration with eps -> 0 returns the pressure advanced by the travel
  time and rescaled by t / |x_d - x_p| (closed form);
* noise-free synthetic pressures of smooth data are inverted to within the
  regularisation error.
"""
import math

import numpy as np
import scipy.linalg

import synthetic as S
from oracle import prep_oracle as R


def test_deconvolution_is_the_tikhonov_minimiser():
    rng = np.random.default_rng(0)
    T, dr = 12, 0.05
    L = R.transform_length(T)
    assert L == 32
    p = rng.standard_normal(T)
    h = rng.standard_normal(T)
    t0 = 0.5 * dr
    eps_rel = 1e-2
    ft = R.deconvolve_detector(p, h, t0, t0, dr, eps_rel)      # delay 0
    C = scipy.linalg.circulant(np.concatenate([dr * h, np.zeros(L - T)]))
    H = np.fft.fft(np.concatenate([dr * h, np.zeros(L - T)]))
    eps = eps_rel * np.max(np.abs(H) ** 2)
    pp = np.concatenate([p, np.zeros(L - T)])
    ref = np.linalg.solve(C.T @ C + eps * np.eye(L), C.T @ pp)[:T]
    assert np.max(np.abs(ft - ref)) < 1e-10 * np.max(np.abs(ref))


def test_integer_shift_is_a_roll():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(16)
    for k in (0, 3, 7):
        y = np.real(np.fft.ifft(R.shift_spectrum(np.fft.fft(x), float(k))))
        assert np.max(np.abs(y - np.roll(x, -k))) < 1e-12


def test_unit_impulse_calibration_advances_and_rescales():
    rng = np.random.default_rng(2)
    D, T, dr, r0 = 3, 20, 0.1, 0.0
    det = np.array([[1.2, 0.0], [0.0, 1.3], [-1.1, 0.2]])
    xp = np.array([0.1, 0.05])
    t = r0 + (np.arange(T) + 0.5) * dr
    dist = np.hypot(det[:, 0] - xp[0], det[:, 1] - xp[1])
    # move the source so that every travel time is a whole number of samples past t0
    j = np.round((dist - t[0]) / dr).astype(int)
    p = rng.standard_normal((D, T))
    pcal = np.zeros((D, T))
    for d in range(D):
        pcal[d, j[d]] = 1.0
    out = np.zeros((D, T))
    for d in range(D):
        ft = R.deconvolve_detector(p[d], pcal[d], t[0] + j[d] * dr, t[0], dr, 1e-14)
        out[d] = t / (t[0] + j[d] * dr) * ft
    for d in range(D):
        # h = the unit impulse at lag 0, times dr: f_t = p / dr
        assert np.max(np.abs(out[d] - t / (t[0] + j[d] * dr) * p[d] / dr)) < 1e-8 * np.max(np.abs(p[d] / dr))


def test_synthetic_round_trip_within_regularisation():
    D, T = 4, 256
    det = S.detectors_full_circle(D, 1.2)
    r0, dr = S.radial_sampling(det, T)
    xp = (0.05, -0.1)
    t = r0 + (np.arange(T) + 0.5) * dr
    f = np.exp(-((t[None, :] - 1.0 - 0.2 * np.arange(D)[:, None]) / 0.15) ** 2)
    # a monopolar (Gaussian) pulse keeps every frequency of the smooth data, so the inverse
    # is exact up to the pulse's truncation and the band-limited shift
    p, pcal = S.pressure_measurement(f, det, xp, r0, dr, width=2 * dr, noise_level=0.0, seed=0, bipolar=False)
    out = R.preprocess(p, pcal, det, xp, r0, dr, eps_rel=1e-8)
    assert np.linalg.norm(out - f) <= 1e-4 * np.linalg.norm(f)
