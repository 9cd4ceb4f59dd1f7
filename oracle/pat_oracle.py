"""Plain FP64 CPU oracle for the preconditioned PDHG reconstruction of photoacoustic
tomography (Boink, Lagerwerf, Steenbergen, van Gils, Manohar, Brune: "A Framework for
Directional and Higher-Order Reconstruction in Photoacoustic Tomography").

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module.  The CUDA library never imports,
links or executes it, and it shares no code, tables or helpers with the CUDA path.
Everything is numpy/scipy in float64, written for readability, not speed.

What it computes (paper section / equation / algorithm in brackets):

* ``forward`` / ``adjoint`` / ``system_matrix``: the discrete circular-mean operator K
  [Sec. 4.2, eq. (K_def); Sec. 3.3.1] and its exact matrix transpose K^T.
* ``grad``/``div`` and ``sym_grad``/``sym_grad_adj``: the finite-difference matrices
  standing in for the gradient and the symmetrised gradient [Sec. 2.1, eq. (min_TGV);
  Sec. 3.3.1 "matrix versions"].
* ``prox_f1_conj``, ``proj_ball``: the dual prox maps [Sec. 3.2].
* ``diag_steps``: the operator-dependent diagonal preconditioners of Pock and Chambolle
  (alpha = 1) cited in Sec. 3.3.2; ``scalar2_steps``: the paper's own two-block rule.
* ``pdhg``: Algorithm 1 (TV) and Algorithm 2 (TGV), plus the directional-TV variant.
* ``duality_gap`` / ``residual``: the validation criteria of Sec. 3.3.3.

Readings where the paper is silent, garbled or inconsistent (each restated beside the
code that uses it):

R1  Discrete K: detector d at x_d, radii r_k = r0 + (k + 1/2) dr (speed of sound 1, so
    time = radius), M quadrature angles phi_m = 2 pi (m + 1/2) / M, points
    x = x_d + r_k (cos phi_m, sin phi_m), bilinear interpolation on pixel centres with
    zero outside the grid, weight 2 pi r_k / M (arc length: eq. (K_def) is a line
    integral over the circle, not a mean).
R2  Gradient: forward differences with unit spacing and zero difference on the last
    row / column (Neumann); div = -grad^T exactly.
R3  Symmetrised gradient: backward differences  d^- = -(d^+)^T, and the symmetric
    2x2 field is stored in orthonormal coordinates (e11, e22, sqrt(2) e12), so the
    pointwise Frobenius norm of the paper's (L^1)^{dxd} term is the Euclidean norm of
    the three stored components and the adjoint is the plain transpose.
R4  F1 is the squared half norm (the square is missing in eq. (PD_TV), present in
    eq. (conj_F1)).
R5  Steps (default): Pock-Chambolle diagonal preconditioning with alpha = 1 on the
    stacked operator A: tau_j = 1 / sum_i |A_ij|, sigma_i = 1 / sum_j |A_ij|.  Dual
    variables that are projected as a pointwise group (r, s) share one sigma, the
    largest admissible for all rows of the group, 1 / (max row sum of the group), so
    the Sigma-weighted prox stays a Euclidean projection.  A zero row imposes no bound
    (any positive sigma is admissible there); an all-zero group or row takes sigma = 1.
R6  theta = 1 (PDHGM).
R7  Duality gap: with G = 0 the paper's D^n is +infinity unless A^T y = 0 exactly, so
    the gap is taken on the box |u| <= U, |v| <= V:  gap = P(x) - D_B(y) with
    P(x) = F(Ax) and D_B(y) = -F*(y) - U ||K^T q - div r||_1 - V ||E^T s - r||_1.
    rel_gap = gap / P(x).  The gap is evaluated on (x^{n+1}, y^{n+1}).
R8  Residual: ||x^{n+1} - x^n||_2 / ||x^n||_2 over the primal variables.
R9  Directional TV (not in this version of the paper): R(u) = ||D_xi grad u||_{1,2},
    D_xi = I - gamma xi xi^T, xi = grad w / sqrt(|grad w|^2 + eta^2).

Parity pins live in tests/test_oracle_pins.py (closed forms, adjoint identities, hand-worked
residual sequences, the direction field of a ramp,
independent solvers, limits).  No function here is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp

REG_TV, REG_TGV, REG_DTV = 0, 1, 2
_SQRT2 = math.sqrt(2.0)


# =============================================================================
# geometry and the circular-mean operator K  [Sec. 3.3.1, Sec. 4.2 eq. (K_def)]
# =============================================================================

@dataclass
class Geometry:
    """Image grid, point detectors and radial / angular sampling (reading R1)."""
    n: int
    det_xy: np.ndarray            # (D, 2) detector positions
    n_t: int                      # number of radius (time) samples T
    r0: float                     # r_k = r0 + (k + 1/2) dr
    dr: float
    quad_m: int                   # quadrature points per circle M
    xmin: float = -1.0
    xmax: float = 1.0
    ymin: float = -1.0
    ymax: float = 1.0

    def __post_init__(self):
        self.det_xy = np.asarray(self.det_xy, dtype=np.float64).reshape(-1, 2)

    @property
    def n_det(self) -> int:
        return self.det_xy.shape[0]

    @property
    def hx(self) -> float:
        return (self.xmax - self.xmin) / self.n

    @property
    def hy(self) -> float:
        return (self.ymax - self.ymin) / self.n

    def radii(self) -> np.ndarray:
        return self.r0 + (np.arange(self.n_t, dtype=np.float64) + 0.5) * self.dr

    def angles(self) -> np.ndarray:
        return 2.0 * math.pi * (np.arange(self.quad_m, dtype=np.float64) + 0.5) / self.quad_m

    def arc_weights(self) -> np.ndarray:
        """Quadrature weight of every point on circle k: its share 2 pi r_k / M of the arc."""
        return 2.0 * math.pi * self.radii() / self.quad_m


def circle_points(g: Geometry, d: int) -> tuple[np.ndarray, np.ndarray]:
    """Quadrature points of all circles around detector d; arrays of shape (T, M)."""
    r = g.radii()[:, None]
    phi = g.angles()[None, :]
    return g.det_xy[d, 0] + r * np.cos(phi), g.det_xy[d, 1] + r * np.sin(phi)


def bilinear_taps(g: Geometry, X: np.ndarray, Y: np.ndarray):
    """The four pixels around each point and their bilinear weights.

    Pixel (ix, iy) has its centre at (xmin + (ix + 1/2) hx, ymin + (iy + 1/2) hy).
    Returns a list of (ix, iy, weight, inside) with ``inside`` marking taps on the grid;
    taps off the grid carry zero image value (reading R1).
    """
    fx = (X - g.xmin) / g.hx - 0.5
    fy = (Y - g.ymin) / g.hy - 0.5
    i0 = np.floor(fx)
    j0 = np.floor(fy)
    ax = fx - i0
    ay = fy - j0
    i0 = i0.astype(np.int64)
    j0 = j0.astype(np.int64)
    taps = []
    for di, dj, wgt in ((0, 0, (1 - ax) * (1 - ay)), (1, 0, ax * (1 - ay)),
                        (0, 1, (1 - ax) * ay), (1, 1, ax * ay)):
        ix = i0 + di
        iy = j0 + dj
        inside = (ix >= 0) & (ix < g.n) & (iy >= 0) & (iy < g.n)
        taps.append((ix, iy, wgt, inside))
    return taps


def forward(g: Geometry, u: np.ndarray) -> np.ndarray:
    """y = K u: circle integrals of the bilinear image, shape (D, T)  [eq. (K_def)]."""
    u = np.asarray(u, dtype=np.float64).reshape(g.n, g.n)
    w = g.arc_weights()
    y = np.zeros((g.n_det, g.n_t))
    for d in range(g.n_det):
        X, Y = circle_points(g, d)
        acc = np.zeros_like(X)
        for ix, iy, wgt, inside in bilinear_taps(g, X, Y):
            vals = u[np.clip(iy, 0, g.n - 1), np.clip(ix, 0, g.n - 1)]
            acc += np.where(inside, wgt * vals, 0.0)
        y[d] = w * acc.sum(axis=1)
    return y


def adjoint(g: Geometry, y: np.ndarray) -> np.ndarray:
    """u = K^T y, the literal transpose of ``forward``'s weights  [Sec. 3.3.1]."""
    y = np.asarray(y, dtype=np.float64).reshape(g.n_det, g.n_t)
    w = g.arc_weights()
    out = np.zeros(g.n * g.n)
    for d in range(g.n_det):
        if not np.any(y[d]):
            continue                      # a zero data row contributes nothing
        X, Y = circle_points(g, d)
        c = np.broadcast_to((w * y[d])[:, None], X.shape)
        for ix, iy, wgt, inside in bilinear_taps(g, X, Y):
            idx = (iy * g.n + ix)[inside]
            out += np.bincount(idx, weights=(c * wgt)[inside], minlength=g.n * g.n)
    return out.reshape(g.n, g.n)


def system_matrix(g: Geometry) -> sp.csr_matrix:
    """K as an explicit sparse matrix (rows d*T + k, columns iy*N + ix).

    The paper precomputes the discrete K once and uses its transpose as the adjoint
    [Sec. 3.3.1]; this builds the same triplets as ``forward``.
    """
    w = g.arc_weights()
    blocks = []
    for d in range(g.n_det):
        X, Y = circle_points(g, d)
        rows_k = np.broadcast_to(np.arange(g.n_t)[:, None], X.shape)
        rr, cc, vv = [], [], []
        for ix, iy, wgt, inside in bilinear_taps(g, X, Y):
            rr.append(rows_k[inside])
            cc.append((iy * g.n + ix)[inside])
            vv.append((w[:, None] * wgt)[inside])
        blk = sp.coo_matrix((np.concatenate(vv), (np.concatenate(rr), np.concatenate(cc))),
                            shape=(g.n_t, g.n * g.n)).tocsr()
        blk.sum_duplicates()
        blocks.append(blk)
    return sp.vstack(blocks, format="csr")


def forward_rows(g: Geometry, u: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Selected entries (d*T + k) of K u, each computed on its own (for large sizes)."""
    u = np.asarray(u, dtype=np.float64).reshape(g.n, g.n)
    r_all = g.radii()
    phi = g.angles()
    out = np.zeros(len(rows))
    for t, row in enumerate(np.asarray(rows)):
        d, k = divmod(int(row), g.n_t)
        X = g.det_xy[d, 0] + r_all[k] * np.cos(phi)
        Y = g.det_xy[d, 1] + r_all[k] * np.sin(phi)
        s = 0.0
        for ix, iy, wgt, inside in bilinear_taps(g, X, Y):
            vals = u[np.clip(iy, 0, g.n - 1), np.clip(ix, 0, g.n - 1)]
            s += float(np.sum(np.where(inside, wgt * vals, 0.0)))
        out[t] = 2.0 * math.pi * r_all[k] / g.quad_m * s
    return out


# =============================================================================
# finite differences  [Sec. 2.1 eqs. (min_TV), (min_TGV); Sec. 3.3.1]
# =============================================================================
# Arrays are (..., N, N) with axis -1 = x (column index ix) and axis -2 = y (row iy).

def dx_fwd(u):
    """Forward difference along x, zero on the last column (reading R2)."""
    out = np.zeros_like(u, dtype=np.float64)
    out[..., :, :-1] = u[..., :, 1:] - u[..., :, :-1]
    return out


def dy_fwd(u):
    out = np.zeros_like(u, dtype=np.float64)
    out[..., :-1, :] = u[..., 1:, :] - u[..., :-1, :]
    return out


def dx_bwd(v):
    """Backward difference along x defined as -(dx_fwd)^T (reading R3)."""
    out = np.zeros_like(v, dtype=np.float64)
    n = v.shape[-1]
    if n == 1:
        return out
    out[..., :, 0] = v[..., :, 0]
    out[..., :, 1:-1] = v[..., :, 1:-1] - v[..., :, :-2]
    out[..., :, -1] = -v[..., :, -2]
    return out


def dy_bwd(v):
    out = np.zeros_like(v, dtype=np.float64)
    n = v.shape[-2]
    if n == 1:
        return out
    out[..., 0, :] = v[..., 0, :]
    out[..., 1:-1, :] = v[..., 1:-1, :] - v[..., :-2, :]
    out[..., -1, :] = -v[..., -2, :]
    return out


def grad(u):
    """grad u = (d_x^+ u, d_y^+ u), shape (2, N, N)."""
    return np.stack([dx_fwd(u), dy_fwd(u)])


def div(p):
    """div p = -grad^T p."""
    return dx_bwd(p[0]) + dy_bwd(p[1])


def sym_grad(v):
    """E v for v = (v1, v2): (d_x^- v1, d_y^- v2, (d_y^- v1 + d_x^- v2)/sqrt 2), shape (3, N, N)."""
    return np.stack([dx_bwd(v[0]), dy_bwd(v[1]), (dy_bwd(v[0]) + dx_bwd(v[1])) / _SQRT2])


def sym_grad_adj(s):
    """E^T s, the transpose of ``sym_grad`` (d_x^-)^T = -d_x^+."""
    return np.stack([-dx_fwd(s[0]) - dy_fwd(s[2]) / _SQRT2,
                     -dy_fwd(s[1]) - dx_fwd(s[2]) / _SQRT2])


def direction_field(w, eta):
    """xi = grad w / sqrt(|grad w|^2 + eta^2)  (reading R9)."""
    gw = grad(np.asarray(w, dtype=np.float64))
    return gw / np.sqrt(gw[0] ** 2 + gw[1] ** 2 + eta * eta)


def dtv_apply(xi, gamma, p):
    """Pointwise D_xi p with D_xi = I - gamma xi xi^T (symmetric, so also its transpose)."""
    dot = xi[0] * p[0] + xi[1] * p[1]
    return np.stack([p[0] - gamma * xi[0] * dot, p[1] - gamma * xi[1] * dot])


def pointwise_norm(p):
    """|p|_2 over the component axis 0."""
    return np.sqrt(np.sum(np.asarray(p) ** 2, axis=0))


# =============================================================================
# proximal maps  [Sec. 3.2]
# =============================================================================

def prox_f1_conj(z, sigma, f):
    """prox of sigma F1^*, F1 = 1/2 ||. - f||^2:  (z - sigma f)/(1 + sigma)  [Sec. 3.2]."""
    return (z - sigma * f) / (1.0 + sigma)


def proj_ball(p, radius):
    """prox of F2^* (and F3^*): radius p / max(radius, |p|_2), pointwise  [Sec. 3.2].

    With radius 0 and p = 0 the formula reads 0/0; the projection onto {0} is 0.
    """
    den = np.maximum(radius, pointwise_norm(p))
    return np.where(den > 0, radius * p / np.where(den > 0, den, 1.0), 0.0)


# =============================================================================
# the saddle-point problem  [Sec. 3.1 eqs. (PD_TV), (PD_TGV)]
# =============================================================================

@dataclass
class Problem:
    """min_u 1/2||K u - f||^2 + alpha R(u) with R = TV, TGV^2_beta or directional TV.

    ``K`` / ``KT`` are callables on (N, N) images and (S,) data vectors; ``k_abs_rows``
    and ``k_abs_cols`` are the row and column sums of |K| (K >= 0 for the circular
    mean, so they are K 1 and K^T 1).
    """
    n: int
    K: Callable
    KT: Callable
    f: np.ndarray
    reg: int = REG_TV
    alpha: float = 0.05
    beta: float = 1.0
    gamma: float = 0.95
    xi: Optional[np.ndarray] = None
    box_u: float = 2.0
    box_v: float = 4.0
    k_abs_rows: Optional[np.ndarray] = None
    k_abs_cols: Optional[np.ndarray] = None

    def __post_init__(self):
        self.f = np.asarray(self.f, dtype=np.float64).reshape(-1)
        if self.reg == REG_DTV and self.xi is None:
            raise ValueError("directional TV needs a direction field xi")


def problem_from_geometry(g: Geometry, f, **kw) -> Problem:
    """Problem whose K is the explicit sparse matrix of ``system_matrix`` (paper Sec. 3.3.1)."""
    Km = system_matrix(g)
    n = g.n
    return Problem(n=n, K=lambda u: Km @ np.asarray(u).reshape(-1),
                   KT=lambda y: (Km.T @ np.asarray(y).reshape(-1)).reshape(n, n),
                   f=f, k_abs_rows=np.asarray(abs(Km).sum(axis=1)).ravel(),
                   k_abs_cols=np.asarray(abs(Km).sum(axis=0)).ravel().reshape(n, n), **kw)


def problem_from_matrix(Km, n: int, f, **kw) -> Problem:
    """Problem with an arbitrary dense or sparse K (used for the K = I denoising pins)."""
    Km = sp.csr_matrix(Km)
    return Problem(n=n, K=lambda u: Km @ np.asarray(u).reshape(-1),
                   KT=lambda y: (Km.T @ np.asarray(y).reshape(-1)).reshape(n, n),
                   f=f, k_abs_rows=np.asarray(abs(Km).sum(axis=1)).ravel(),
                   k_abs_cols=np.asarray(abs(Km).sum(axis=0)).ravel().reshape(n, n), **kw)


def regulariser_operator(pb: Problem) -> sp.csr_matrix:
    """The non-K rows of the stacked operator A as an explicit sparse matrix.

    Built from Kronecker products of 1-D difference matrices, independently of the
    array functions above.  Unknowns: u (N^2) and, for TGV, v1, v2 (N^2 each), all
    row-major.  Rows: TV r1, r2; TGV r1, r2, s11, s22, s12; dTV (D_xi grad) rows.
    """
    n = pb.n
    I = sp.identity(n, format="csr")
    Dp = sp.diags([-np.ones(n), np.ones(n - 1)], [0, 1], shape=(n, n), format="lil")
    Dp[n - 1, :] = 0                      # Neumann: no difference on the last index
    Dp = Dp.tocsr()
    Dm = (-Dp.T).tocsr()                  # backward difference -(D^+)^T
    Gx = sp.kron(I, Dp, format="csr")     # x varies fastest (columns)
    Gy = sp.kron(Dp, I, format="csr")
    if pb.reg == REG_TV:
        return sp.vstack([Gx, Gy], format="csr")
    if pb.reg == REG_DTV:
        xi = pb.xi.reshape(2, -1)
        d11 = sp.diags(1.0 - pb.gamma * xi[0] * xi[0])
        d12 = sp.diags(-pb.gamma * xi[0] * xi[1])
        d22 = sp.diags(1.0 - pb.gamma * xi[1] * xi[1])
        return sp.vstack([d11 @ Gx + d12 @ Gy, d12 @ Gx + d22 @ Gy], format="csr")
    Ex = sp.kron(I, Dm, format="csr")
    Ey = sp.kron(Dm, I, format="csr")
    I2 = sp.identity(n * n, format="csr")
    Z = sp.csr_matrix((n * n, n * n))
    return sp.bmat([[Gx, -I2, None],
                    [Gy, None, -I2],
                    [None, Ex, Z],
                    [None, Z, Ey],
                    [None, Ey / _SQRT2, Ex / _SQRT2]], format="csr")


@dataclass
class Steps:
    sig_q: np.ndarray
    sig_r: np.ndarray
    tau_u: np.ndarray
    sig_s: Optional[np.ndarray] = None
    tau_v: Optional[np.ndarray] = None


def diag_steps(pb: Problem) -> Steps:
    """Pock-Chambolle diagonal preconditioners, alpha = 1 (Sec. 3.3.2, reading R5).

    sigma_i = 1 / sum_j |A_ij| and tau_j = 1 / sum_i |A_ij| for the stacked
    A = (K; B) with B from ``regulariser_operator``.  Pointwise groups (r: 2 rows,
    s: 3 rows at one pixel) share sigma = 1 / (largest row sum in the group).
    """
    n2 = pb.n * pb.n
    B = abs(regulariser_operator(pb))
    b_rows = np.asarray(B.sum(axis=1)).ravel()
    b_cols = np.asarray(B.sum(axis=0)).ravel()
    krow = np.asarray(pb.k_abs_rows, dtype=np.float64).ravel()
    kcol = np.asarray(pb.k_abs_cols, dtype=np.float64).ravel()

    def inv(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where(x > 0, 1.0 / np.where(x > 0, x, 1.0), 1.0)

    def group_sigma(sums):
        # largest sigma admissible for every row of the group: 1 / max row sum; rows
        # whose sum is zero impose no bound (1 when the whole group is zero)
        return inv(np.max(sums, axis=0))

    sig_q = inv(krow)
    g = 2 if pb.reg != REG_TGV else 5
    rows = b_rows.reshape(g, pb.n, pb.n)
    sig_r = group_sigma(rows[0:2])
    sig_s = group_sigma(rows[2:5]) if pb.reg == REG_TGV else None
    tau_u = inv(kcol + b_cols[:n2]).reshape(pb.n, pb.n)
    tau_v = inv(b_cols[n2:]).reshape(2, pb.n, pb.n) if pb.reg == REG_TGV else None
    return Steps(sig_q=sig_q, sig_r=sig_r, tau_u=tau_u, sig_s=sig_s, tau_v=tau_v)


def balanced_steps(st: Steps, ratio: float) -> Steps:
    """The primal-dual balance of a step choice: every primal step times ``ratio`` and
    every dual step divided by it.  ||Sigma^1/2 A T^1/2|| is unchanged, so the
    convergence condition of Sec. 3.3.2 still holds."""
    def sc(a, m):
        return None if a is None else np.asarray(a, dtype=np.float64) * m
    return Steps(sig_q=sc(st.sig_q, 1.0 / ratio), sig_r=sc(st.sig_r, 1.0 / ratio), tau_u=sc(st.tau_u, ratio),
                 sig_s=sc(st.sig_s, 1.0 / ratio), tau_v=sc(st.tau_v, ratio))


def power_norm(apply, apply_t, x0, iters: int) -> float:
    """Largest singular value by power iteration on apply_t(apply(.)) from x0."""
    x = np.asarray(x0, dtype=np.float64)
    x = x / np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = apply_t(apply(x))
        lam = float(np.linalg.norm(y))
        if lam == 0.0:
            return 0.0
        x = y / lam
    return math.sqrt(lam)


def power_start(size: int) -> np.ndarray:
    """Deterministic start vector x_j = 1 + sin(0.7 j + 0.3) / 2 for the power iteration."""
    j = np.arange(size, dtype=np.float64)
    return 1.0 + 0.5 * np.sin(0.7 * j + 0.3)


def scalar2_steps(pb: Problem, power_iters: int = 100, safety: float = 0.99) -> Steps:
    """The paper's two-block scalar steps (Sec. 3.3.2): sigma_1 tau L1^2 < 1/4,
    sigma_2 tau L2^2 < 1/4, with L1 = ||K||, L2 = ||B|| by power iteration.

    tau is free in the paper; tau = 1/L1 is taken, sigma_i = safety / (4 tau L_i^2).
    """
    n = pb.n
    L1 = power_norm(lambda x: pb.K(x.reshape(n, n)), lambda y: np.asarray(pb.KT(y)).reshape(-1),
                    power_start(n * n), power_iters)
    B = regulariser_operator(pb)
    L2 = power_norm(lambda x: B @ x, lambda y: B.T @ y, power_start(B.shape[1]), power_iters)
    tau = 1.0 / L1
    s1 = safety / (4.0 * tau * L1 * L1)
    s2 = safety / (4.0 * tau * L2 * L2)
    S = pb.f.size
    one = np.ones((n, n))
    st = Steps(sig_q=np.full(S, s1), sig_r=s2 * one, tau_u=tau * one)
    if pb.reg == REG_TGV:
        st.sig_s = s2 * one
        st.tau_v = tau * np.ones((2, n, n))
    return st


# =============================================================================
# objective, duality gap and residual  [Sec. 3.3.3]
# =============================================================================

def regulariser(pb: Problem, u, v=None) -> float:
    """R(u) without alpha: TV, TGV (first + beta * second order term) or dTV."""
    if pb.reg == REG_TV:
        return float(np.sum(pointwise_norm(grad(u))))
    if pb.reg == REG_DTV:
        return float(np.sum(pointwise_norm(dtv_apply(pb.xi, pb.gamma, grad(u)))))
    return float(np.sum(pointwise_norm(grad(u) - v)) + pb.beta * np.sum(pointwise_norm(sym_grad(v))))


def primal_objective(pb: Problem, u, v=None) -> float:
    """P(x) = 1/2 ||K u - f||^2 + alpha R(u)  [eq. (min_prob)]."""
    res = np.asarray(pb.K(u)).reshape(-1) - pb.f
    return 0.5 * float(res @ res) + pb.alpha * regulariser(pb, u, v)


def duality_gap(pb: Problem, u, q, r, v=None, s=None, KTq=None) -> dict:
    """Box-restricted duality gap (reading R7); dual variables must be feasible."""
    primal = primal_objective(pb, u, v)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    f1c = 0.5 * float(q @ q) + float(q @ pb.f)            # F1^*(q) [eq. (conj_F1)]
    if KTq is None:
        KTq = np.asarray(pb.KT(q)).reshape(pb.n, pb.n)
    if pb.reg == REG_DTV:
        gu = KTq - div(dtv_apply(pb.xi, pb.gamma, r))
    else:
        gu = KTq - div(r)
    dual = -f1c - pb.box_u * float(np.sum(np.abs(gu)))
    # the part of the gap that measures A^T y != 0 (primal stationarity, G = 0):
    # U ||A_u^T y||_1 + V ||A_v^T y||_1 + <x, A^T y>; the rest is the Fenchel-Young gap
    # F(Ax) + F^*(y) - <Ax, y> >= 0 of the dual variables
    stat = pb.box_u * float(np.sum(np.abs(gu))) + float(np.sum(u * gu))
    if pb.reg == REG_TGV:
        gv = sym_grad_adj(s) - r
        dual -= pb.box_v * float(np.sum(np.abs(gv)))
        stat += pb.box_v * float(np.sum(np.abs(gv))) + float(np.sum(v * gv))
    gap = primal - dual
    return {"primal": primal, "dual": dual, "gap": gap, "stationarity": stat,
            "rel_gap": gap / primal if primal > 0 else (0.0 if gap == 0 else math.inf)}


def _cone_distance(g, p, radius):
    """Pointwise distance of g from the normal cone of the radius-ball at p (p inside the
    ball: the cone is {0}; p on the sphere: the ray through p)."""
    npn = pointwise_norm(p)
    on = npn >= radius * (1.0 - 1e-6)
    lam = np.where(on, np.maximum(0.0, np.sum(g * p, axis=0) / np.where(npn > 0, npn, 1.0)), 0.0)
    return np.sqrt(np.maximum(np.sum(g * g, axis=0) - lam * lam, 0.0))


def pd_residuals(pb: Problem, u, q, r, v=None, s=None, KTq=None) -> tuple[float, float]:
    """Primal and dual residuals of Goldstein, Li, Yuan, Esser and Baraniuk (2015) at a
    state, in the L1 norm.  Primal: |A^T y|_1 (G = 0, so 0 = A^T y at a solution).  Dual:
    the distance of A x from dF^*(y): |q - (K u - f)|_1 for the data term, and for the
    ball-constrained duals the distance of their argument from the normal cone of the
    ball at r and s."""
    n = pb.n
    if KTq is None:
        KTq = np.asarray(pb.KT(q)).reshape(n, n)
    rr = dtv_apply(pb.xi, pb.gamma, r) if pb.reg == REG_DTV else r
    prim = float(np.sum(np.abs(KTq - div(rr))))
    Ku = np.asarray(pb.K(u)).reshape(-1)
    dual = float(np.sum(np.abs(np.asarray(q).reshape(-1) - (Ku - pb.f))))
    g = grad(u)
    if pb.reg == REG_DTV:
        g = dtv_apply(pb.xi, pb.gamma, g)
    if pb.reg == REG_TGV:
        g = g - v
        prim += float(np.sum(np.abs(sym_grad_adj(s) - r)))
        dual += float(np.sum(_cone_distance(sym_grad(v), s, pb.alpha * pb.beta)))
    dual += float(np.sum(_cone_distance(g, r, pb.alpha)))
    return prim, dual


# Adaptive primal-dual balance (residual balancing after Goldstein et al. 2015): at every
# gap evaluation, when the primal residual exceeds the dual one by more than BALANCE_DEAD
# the primal steps grow (s up), when the dual one dominates they shrink.  s moves by the
# square root of the residual ratio, at most a factor BALANCE_MAX_STEP, with an exponent
# that decays by BALANCE_DECAY per adjustment so that s settles.
BALANCE_DEAD = 2.0
BALANCE_MAX_STEP = 2.0
BALANCE_DECAY = 0.97
BALANCE_RANGE = (1e-3, 1e3)


def balance_update(ratio: float, primal_res: float, dual_res: float, n_adjust: int) -> tuple[float, int]:
    """One adaptive-balance decision; returns (new s, new adjustment count)."""
    if not (primal_res > 0 and dual_res > 0):
        return ratio, n_adjust
    rho = primal_res / dual_res
    if 1.0 / BALANCE_DEAD <= rho <= BALANCE_DEAD:
        return ratio, n_adjust
    f = min(max(math.sqrt(rho), 1.0 / BALANCE_MAX_STEP), BALANCE_MAX_STEP)
    new = ratio * f ** (BALANCE_DECAY ** n_adjust)
    return min(max(new, BALANCE_RANGE[0]), BALANCE_RANGE[1]), n_adjust + 1


def residual(x_new: list, x_old: list) -> float:
    """||x^{n+1} - x^n||_2 / ||x^n||_2 over all primal arrays (reading R8)."""
    num = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(x_new, x_old)))
    den = math.sqrt(sum(float(np.sum(b ** 2)) for b in x_old))
    if den > 0:
        return num / den
    return 0.0 if num == 0 else math.inf


# =============================================================================
# PDHGM  [Sec. 3.3, Algorithm 1 (TV), Algorithm 2 (TGV)]
# =============================================================================

@dataclass
class Result:
    u: np.ndarray
    v: Optional[np.ndarray]
    q: np.ndarray
    r: np.ndarray
    s: Optional[np.ndarray]
    iters_done: int
    gap: dict = field(default_factory=dict)
    residual: float = math.nan
    history: list = field(default_factory=list)
    step_ratio: float = 1.0
    ubar: Optional[np.ndarray] = None
    vbar: Optional[np.ndarray] = None


def pdhg(pb: Problem, iters: int, steps: Optional[Steps] = None, theta: float = 1.0,
         tol: float = 0.0, gap_every: int = 0, x0: Optional[dict] = None,
         y0: Optional[dict] = None, xbar0: Optional[dict] = None, final_gap: bool = True,
         step_ratio: float = 1.0, adapt: bool = False) -> Result:
    """Preconditioned PDHGM, one iteration per step of Algorithm 1 / Algorithm 2.

    Iterates start at zero (the initialisation of Algorithms 1 and 2) unless
    ``x0`` = {u, v} / ``y0`` = {q, r, s} are given; the extrapolated point starts at
    ``xbar0`` = {u, v} if given, else at x^0.  ``final_gap`` = False skips the gap
    evaluation after the last iteration when ``gap_every`` does not ask for it.  When ``gap_every`` > 0 the gap is evaluated after every
    ``gap_every``-th iteration (and after the last one); with ``tol`` > 0 the loop stops
    at the first evaluation with rel_gap <= tol.
    """
    n = pb.n
    st0 = steps if steps is not None else diag_steps(pb)
    ratio, n_adjust = float(step_ratio), 0
    st = balanced_steps(st0, ratio)
    tgv = pb.reg == REG_TGV
    u = np.zeros((n, n)) if x0 is None else np.array(x0["u"], dtype=np.float64).reshape(n, n)
    v = None
    if tgv:
        v = np.zeros((2, n, n)) if x0 is None or x0.get("v") is None else \
            np.array(x0["v"], dtype=np.float64).reshape(2, n, n)
    q = np.zeros(pb.f.size) if y0 is None else np.array(y0["q"], dtype=np.float64).reshape(-1)
    r = np.zeros((2, n, n)) if y0 is None else np.array(y0["r"], dtype=np.float64).reshape(2, n, n)
    s = None
    if tgv:
        s = np.zeros((3, n, n)) if y0 is None or y0.get("s") is None else \
            np.array(y0["s"], dtype=np.float64).reshape(3, n, n)
    ubar = u.copy() if xbar0 is None else np.array(xbar0["u"], dtype=np.float64).reshape(n, n)
    vbar = None
    if tgv:
        vbar = v.copy() if xbar0 is None or xbar0.get("v") is None else \
            np.array(xbar0["v"], dtype=np.float64).reshape(2, n, n)
    out = Result(u=u, v=v, q=q, r=r, s=s, iters_done=0, step_ratio=ratio)
    for it in range(iters):
        # dual steps
        q = prox_f1_conj(q + st.sig_q * np.asarray(pb.K(ubar)).reshape(-1), st.sig_q, pb.f)
        if pb.reg == REG_TV:
            r = proj_ball(r + st.sig_r * grad(ubar), pb.alpha)
        elif pb.reg == REG_DTV:
            r = proj_ball(r + st.sig_r * dtv_apply(pb.xi, pb.gamma, grad(ubar)), pb.alpha)
        else:
            r = proj_ball(r + st.sig_r * (grad(ubar) - vbar), pb.alpha)
            s = proj_ball(s + st.sig_s * sym_grad(vbar), pb.alpha * pb.beta)
        # primal steps (prox of G = 0 is the identity)
        KTq = np.asarray(pb.KT(q)).reshape(n, n)
        if pb.reg == REG_DTV:
            u_new = u - st.tau_u * (KTq - div(dtv_apply(pb.xi, pb.gamma, r)))
        else:
            u_new = u - st.tau_u * (KTq - div(r))
        if tgv:
            v_new = v - st.tau_v * (sym_grad_adj(s) - r)
        # extrapolation
        ubar = u_new + theta * (u_new - u)
        if tgv:
            vbar = v_new + theta * (v_new - v)
        x_old = [u] + ([v] if tgv else [])
        u = u_new
        if tgv:
            v = v_new
        done = it + 1
        check = (gap_every > 0 and done % gap_every == 0) or (final_gap and done == iters)
        if check:
            gp = duality_gap(pb, u, q, r, v, s, KTq=KTq)
            res = residual([u] + ([v] if tgv else []), x_old)
            out.history.append((done, gp["gap"], gp["rel_gap"], res))
            out.gap, out.residual = gp, res
            if adapt:
                pres, dres = pd_residuals(pb, u, q, r, v, s, KTq=KTq)
                ratio, n_adjust = balance_update(ratio, pres, dres, n_adjust)
                st = balanced_steps(st0, ratio)
                out.step_ratio = ratio
            if tol > 0 and gp["rel_gap"] <= tol:
                out.u, out.v, out.q, out.r, out.s, out.iters_done = u, v, q, r, s, done
                out.ubar, out.vbar = ubar, vbar
                return out
        out.iters_done = done
    out.u, out.v, out.q, out.r, out.s = u, v, q, r, s
    out.ubar, out.vbar = ubar, vbar
    return out
