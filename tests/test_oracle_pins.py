"""Pins for the FP64 oracle: checks against what the mathematics fixes, never against the
oracle's own formulas retyped.

* K: the exact circle-disc arc length (closed form, stored fixture), the row sum 2 pi r
  of circles inside the grid, a dense matrix built entry by entry from hat functions.
* K^T: the adjoint identity and agreement with the explicit sparse transpose.
* grad/div, E/E^T: adjoint identities, ramps and quadratics with known differences,
  agreement with an independent Kronecker-product construction.
* prox maps: Moreau decomposition with independently written primal proxes, and
  brute-force minimisation.
* PDHG: ROF and directional-TV denoising against FISTA on the dual, TGV denoising
  against ADMM, the alpha -> infinity constant limit, the alpha = 0 least-squares limit.
* steps: ||Sigma^1/2 A T^1/2|| <= 1 by dense SVD.
* gap: weak duality on random feasible pairs, zero at a known saddle point.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _geom(n=8, n_det=3, n_t=6, m=16, radius=1.2, seed=0):
    ang = 2 * math.pi * (np.arange(n_det) + 0.1 * seed) / n_det
    det = np.stack([radius * np.cos(ang), radius * np.sin(ang)], 1)
    rmax = radius + math.sqrt(2.0)
    return O.Geometry(n=n, det_xy=det, n_t=n_t, r0=0.0, dr=rmax / n_t, quad_m=m)


def _hat(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


# ---------------------------------------------------------------------------
# K
# ---------------------------------------------------------------------------

def _disc_arc_integral(det, r, cx, cy, rho, amp):
    """Exact integral of amp * 1_{disc} over the circle |x - det| = r (arc length inside)."""
    dc = math.hypot(det[0] - cx, det[1] - cy)
    if dc + r <= rho:
        return amp * 2 * math.pi * r
    if r + rho <= dc or dc + rho <= r:
        return 0.0
    c = (dc * dc + r * r - rho * rho) / (2 * dc * r)
    return amp * 2 * r * math.acos(max(-1.0, min(1.0, c)))


def test_golden_disc_arc_lengths_match_closed_form():
    with open(os.path.join(HERE, "golden", "disc_arc_lengths.json")) as fh:
        gold = json.load(fh)
    for case in gold["cases"]:
        val = _disc_arc_integral(case["det"], case["r"], *case["disc"])
        assert abs(val - case["value"]) <= 1e-12 * max(1.0, abs(case["value"]))


def test_K_converges_to_disc_arc_lengths():
    """Discrete K of a finely rasterised disc approaches the exact arc length, O(h)."""
    with open(os.path.join(HERE, "golden", "disc_arc_lengths.json")) as fh:
        gold = json.load(fh)
    cx, cy, rho, amp = gold["phantom"]
    det = np.array(gold["detectors"])
    radii = np.array(gold["radii"])
    errs = []
    for n in (128, 512):
        # pixel averages of the disc (16x16 supersampling per pixel)
        ss = 16
        h = 2.0 / n
        sub = (np.arange(ss) + 0.5) / ss
        c = (-1 + (np.arange(n)[:, None] + sub[None, :]) * h).reshape(-1)
        X, Y = np.meshgrid(c, c)
        img = amp * (((X - cx) ** 2 + (Y - cy) ** 2) <= rho ** 2)
        img = img.reshape(n, ss, n, ss).mean(axis=(1, 3))
        dr = radii[1] - radii[0]
        g = O.Geometry(n=n, det_xy=det, n_t=len(radii), r0=radii[0] - 0.5 * dr, dr=dr,
                       quad_m=8192)
        y = O.forward(g, img)
        want = np.array([[c_["value"] for c_ in gold["cases"] if c_["d"] == d]
                         for d in range(len(det))])
        errs.append(np.max(np.abs(y - want)) / np.max(np.abs(want)))
    assert errs[1] < 0.6 * errs[0]
    assert errs[1] < 5e-3


def test_K_quadrature_of_analytic_disc_converges_in_M():
    """The angular quadrature (weights 2 pi r / M at midpoints) applied to the analytic
    indicator converges to the exact arc length as M grows."""
    det = np.array([1.2, 0.0])
    cx, cy, rho = 0.1, -0.2, 0.4
    for r in (0.9, 1.2, 1.5):
        exact = _disc_arc_integral(det, r, cx, cy, rho, 1.0)
        errs = []
        for m in (512, 8192):
            phi = 2 * math.pi * (np.arange(m) + 0.5) / m
            X = det[0] + r * np.cos(phi)
            Y = det[1] + r * np.sin(phi)
            val = 2 * math.pi * r / m * np.sum(((X - cx) ** 2 + (Y - cy) ** 2) <= rho ** 2)
            errs.append(abs(val - exact))
        assert errs[1] <= errs[0] + 1e-12
        assert errs[1] <= 2 * 2 * math.pi * r / 8192 + 1e-12


def test_K_row_sums_are_circumference_inside_grid():
    """Bilinear weights form a partition of unity inside the pixel-centre hull, so a circle
    lying there integrates the constant image exactly: (K 1)_{d,k} = 2 pi r_k."""
    n = 32
    det = np.array([[0.05, -0.1], [-0.2, 0.15]])
    g = O.Geometry(n=n, det_xy=det, n_t=20, r0=0.0, dr=0.04, quad_m=96)
    y = O.forward(g, np.ones((n, n)))
    r = g.radii()
    hull = 1.0 - 0.5 * g.hx - 1e-9
    for d in range(2):
        for k in range(g.n_t):
            if max(abs(det[d, 0]) + r[k], abs(det[d, 1]) + r[k]) < hull:
                assert abs(y[d, k] - 2 * math.pi * r[k]) < 1e-12
    # and circles entirely off the extended grid give zero
    far = O.Geometry(n=8, det_xy=np.array([[5.0, 5.0]]), n_t=4, r0=0.0, dr=0.5, quad_m=32)
    assert np.all(O.forward(far, np.ones((8, 8))) == 0.0)


def test_K_dense_bruteforce_entry_by_entry():
    """Tiny K built from tensor-product hat functions (a second, independent way of
    writing bilinear interpolation on pixel centres with zero outside the grid)."""
    g = _geom(n=4, n_det=2, n_t=3, m=8)
    D, T, N, M = g.n_det, g.n_t, g.n, g.quad_m
    dense = np.zeros((D * T, N * N))
    for d in range(D):
        for k in range(T):
            r = (k + 0.5) * g.dr
            for m in range(M):
                phi = 2 * math.pi * (m + 0.5) / M
                x = g.det_xy[d, 0] + r * math.cos(phi)
                y = g.det_xy[d, 1] + r * math.sin(phi)
                for iy in range(N):
                    for ix in range(N):
                        cx = -1 + (ix + 0.5) * g.hx
                        cy = -1 + (iy + 0.5) * g.hy
                        dense[d * T + k, iy * N + ix] += (2 * math.pi * r / M) * \
                            _hat((x - cx) / g.hx) * _hat((y - cy) / g.hy)
    assert np.abs(dense).sum() > 0
    Km = O.system_matrix(g).toarray()
    np.testing.assert_allclose(Km, dense, rtol=0, atol=1e-13)
    u = np.random.default_rng(1).standard_normal((N, N))
    np.testing.assert_allclose(O.forward(g, u).ravel(), dense @ u.ravel(), rtol=0, atol=1e-12)
    rows = np.array([0, 3, 5])
    np.testing.assert_allclose(O.forward_rows(g, u, rows), (dense @ u.ravel())[rows], atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_K_adjoint_identity(seed):
    g = _geom(n=13, n_det=5, n_t=17, m=40, seed=seed)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((g.n, g.n))
    y = rng.standard_normal((g.n_det, g.n_t))
    lhs = float(np.sum(O.forward(g, u) * y))
    rhs = float(np.sum(u * O.adjoint(g, y)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    Km = O.system_matrix(g)
    np.testing.assert_allclose(O.adjoint(g, y).ravel(), Km.T @ y.ravel(), atol=1e-12)


def test_K_is_nonnegative():
    Km = O.system_matrix(_geom(n=9, n_det=4, n_t=10, m=24))
    assert Km.data.min() >= 0.0


# ---------------------------------------------------------------------------
# finite differences
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 7])
def test_grad_div_and_sym_grad_adjoints(n):
    rng = np.random.default_rng(n)
    u = rng.standard_normal((n, n))
    p = rng.standard_normal((2, n, n))
    assert abs(np.sum(O.grad(u) * p) + np.sum(u * O.div(p))) < 1e-12
    v = rng.standard_normal((2, n, n))
    s = rng.standard_normal((3, n, n))
    assert abs(np.sum(O.sym_grad(v) * s) - np.sum(v * O.sym_grad_adj(s))) < 1e-12


def test_ramp_and_quadratic_differences():
    n = 6
    iy, ix = np.mgrid[0:n, 0:n].astype(float)
    g = O.grad(3.0 * ix - 2.0 * iy)
    assert np.all(g[0][:, :-1] == 3.0) and np.all(g[0][:, -1] == 0.0)
    assert np.all(g[1][:-1, :] == -2.0) and np.all(g[1][-1, :] == 0.0)
    # interior backward differences of quadratics: x^2 - (x-1)^2 = 2x - 1
    e = O.sym_grad(np.stack([ix ** 2, iy ** 2]))
    assert np.allclose(e[0][:, 1:-1], 2 * ix[:, 1:-1] - 1)
    assert np.allclose(e[1][1:-1, :], 2 * iy[1:-1, :] - 1)
    # mixed term of (x*y, 0): d_y^-(x y) = x, scaled by 1/sqrt 2
    e2 = O.sym_grad(np.stack([ix * iy, np.zeros_like(ix)]))
    assert np.allclose(e2[2][1:-1, :], ix[1:-1, :] / math.sqrt(2))
    # |E v| is the Frobenius norm of [[a, c], [c, b]] with c = (d_y v1 + d_x v2)/2
    v = np.random.default_rng(3).standard_normal((2, n, n))
    e3 = O.sym_grad(v)
    a, b = O.dx_bwd(v[0]), O.dy_bwd(v[1])
    c = 0.5 * (O.dy_bwd(v[0]) + O.dx_bwd(v[1]))
    assert np.allclose(O.pointwise_norm(e3), np.sqrt(a * a + b * b + 2 * c * c))


@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV, O.REG_DTV])
def test_kronecker_operator_matches_array_operators(reg):
    n = 5
    rng = np.random.default_rng(reg)
    xi = rng.standard_normal((2, n, n))
    xi /= np.sqrt(xi[0] ** 2 + xi[1] ** 2 + 0.1)
    pb = O.Problem(n=n, K=None, KT=None, f=np.zeros(1), reg=reg, xi=xi, gamma=0.7)
    B = O.regulariser_operator(pb)
    u = rng.standard_normal((n, n))
    if reg == O.REG_TV:
        want = O.grad(u).ravel()
        got = B @ u.ravel()
    elif reg == O.REG_DTV:
        want = O.dtv_apply(xi, 0.7, O.grad(u)).ravel()
        got = B @ u.ravel()
    else:
        v = rng.standard_normal((2, n, n))
        want = np.concatenate([(O.grad(u) - v).ravel(), O.sym_grad(v).ravel()])
        got = B @ np.concatenate([u.ravel(), v.ravel()])
    np.testing.assert_allclose(got, want, atol=1e-12)


# ---------------------------------------------------------------------------
# prox maps
# ---------------------------------------------------------------------------

def test_prox_f1_conj_moreau_and_bruteforce():
    rng = np.random.default_rng(0)
    z, f = rng.standard_normal(50), rng.standard_normal(50)
    sig = rng.uniform(0.01, 5.0, 50)
    p = O.prox_f1_conj(z, sig, f)
    # Moreau: prox_{sig F*}(z) = z - sig prox_{F/sig}(z/sig), prox of F/sig for
    # F = 1/2|.-f|^2 is (sig x + f)/(sig + 1)
    x = z / sig
    np.testing.assert_allclose(p, z - sig * (sig * x + f) / (sig + 1), atol=1e-12)
    # brute force on a fine grid for a few entries: F*(y) = y^2/2 + y f
    for i in range(5):
        grid = np.linspace(p[i] - 1, p[i] + 1, 200001)
        obj = 0.5 * (grid - z[i]) ** 2 + sig[i] * (0.5 * grid ** 2 + grid * f[i])
        assert abs(grid[np.argmin(obj)] - p[i]) < 2e-5


def test_proj_ball_moreau_with_group_soft_threshold():
    rng = np.random.default_rng(1)
    pts = rng.standard_normal((3, 40)) * 2
    alpha = 0.7
    # primal prox of alpha |.|_2 is group soft thresholding
    nrm = np.sqrt(np.sum(pts ** 2, axis=0))
    soft = pts * np.maximum(0.0, 1.0 - alpha / nrm)
    np.testing.assert_allclose(O.proj_ball(pts, alpha), pts - soft, atol=1e-12)
    proj = O.proj_ball(pts, alpha)
    assert np.all(np.sqrt(np.sum(proj ** 2, 0)) <= alpha + 1e-12)
    # no point of the ball is closer (random sampling)
    for j in range(5):
        cand = rng.standard_normal((3, 2000))
        cand *= alpha * rng.uniform(0, 1, 2000) ** (1 / 3) / np.sqrt(np.sum(cand ** 2, 0))
        d_best = np.sum((proj[:, j] - pts[:, j]) ** 2)
        assert np.all(np.sum((cand - pts[:, [j]]) ** 2, 0) >= d_best - 1e-12)


# ---------------------------------------------------------------------------
# independent solvers for the pins of PDHG
# ---------------------------------------------------------------------------

def _kron_grad(n):
    I = sp.identity(n, format="csr")
    Dp = sp.diags([-np.ones(n), np.ones(n - 1)], [0, 1], shape=(n, n), format="lil")
    Dp[n - 1, :] = 0
    Dp = Dp.tocsr()
    return sp.kron(I, Dp, format="csr"), sp.kron(Dp, I, format="csr"), Dp


def _fista_rof_dual(f, alpha, iters, pointwise_mat=None):
    """min_u 1/2||u - f||^2 + alpha ||M grad u||_{1,2} by FISTA on the dual
    max_{|p|<=alpha} -1/2||f - G^T M p||^2 ...; u = f - G^T M^T p (M symmetric 2x2 field)."""
    n = f.shape[0]
    Gx, Gy, _ = _kron_grad(n)
    G = sp.vstack([Gx, Gy], format="csr")
    if pointwise_mat is not None:
        m11, m12, m22 = (a.ravel() for a in pointwise_mat)
        Mm = sp.bmat([[sp.diags(m11), sp.diags(m12)], [sp.diags(m12), sp.diags(m22)]], format="csr")
        G = Mm @ G
    L = 8.0  # ||grad||^2 <= 8 with unit spacing; |M| <= 1 for D_xi with |xi| < 1
    fv = f.ravel()
    p = np.zeros(G.shape[0])
    z = p.copy()
    t = 1.0
    for _ in range(iters):
        u = fv - G.T @ z
        grad_p = -(G @ u)
        pn = z - grad_p / L
        pn2 = pn.reshape(2, -1)
        nrm = np.sqrt(np.sum(pn2 ** 2, 0))
        pn = (pn2 * (alpha / np.maximum(alpha, nrm))).ravel()
        tn = 0.5 * (1 + math.sqrt(1 + 4 * t * t))
        z = pn + (t - 1) / tn * (pn - p)
        p, t = pn, tn
    return (fv - G.T @ p).reshape(n, n)


def _admm_tgv_denoise(f, alpha, beta, iters, rho=1.0):
    """min_{u,v} 1/2||u-f||^2 + alpha||grad u - v||_{1,2} + alpha beta||E v||_{1,F} by ADMM
    with the splitting z = (grad u - v, E v) and exact dense linear solves."""
    n = f.shape[0]
    pb = O.Problem(n=n, K=None, KT=None, f=np.zeros(1), reg=O.REG_TGV)
    B = O.regulariser_operator(pb).toarray()
    nx = B.shape[1]
    n2 = n * n
    P = np.zeros((nx, nx))
    P[:n2, :n2] = np.eye(n2)
    rhs0 = np.zeros(nx)
    rhs0[:n2] = f.ravel()
    Amat = P + rho * B.T @ B
    Ainv = np.linalg.inv(Amat)
    z = np.zeros(B.shape[0])
    lam = np.zeros_like(z)
    x = np.zeros(nx)
    for _ in range(iters):
        x = Ainv @ (rhs0 + rho * B.T @ (z - lam))
        bx = B @ x
        w = bx + lam
        w1 = w[:2 * n2].reshape(2, n2)
        w2 = w[2 * n2:].reshape(3, n2)
        n1 = np.sqrt(np.sum(w1 ** 2, 0))
        n2_ = np.sqrt(np.sum(w2 ** 2, 0))
        z1 = w1 * np.maximum(0, 1 - (alpha / rho) / np.maximum(n1, 1e-300))
        z2 = w2 * np.maximum(0, 1 - (alpha * beta / rho) / np.maximum(n2_, 1e-300))
        z = np.concatenate([z1.ravel(), z2.ravel()])
        lam = lam + bx - z
    return x[:n2].reshape(n, n)


def _denoise_problem(f, reg, alpha, **kw):
    n = f.shape[0]
    return O.problem_from_matrix(sp.identity(n * n), n, f.ravel(), reg=reg, alpha=alpha, **kw)


def test_pdhg_rof_matches_fista_dual():
    rng = np.random.default_rng(5)
    f = (rng.uniform(size=(6, 6)) > 0.5) + 0.1 * rng.standard_normal((6, 6))
    pb = _denoise_problem(f, O.REG_TV, 0.15)
    res = O.pdhg(pb, 6000)
    ref = _fista_rof_dual(f, 0.15, 40000)
    np.testing.assert_allclose(res.u, ref, atol=2e-6)


def test_pdhg_dtv_denoise_matches_fista_dual_and_gamma0_is_tv():
    rng = np.random.default_rng(6)
    n = 6
    f = (rng.uniform(size=(n, n)) > 0.5) + 0.1 * rng.standard_normal((n, n))
    xi = rng.standard_normal((2, n, n))
    xi /= np.sqrt(xi[0] ** 2 + xi[1] ** 2 + 0.3)
    gamma = 0.8
    pb = _denoise_problem(f, O.REG_DTV, 0.15, xi=xi, gamma=gamma)
    res = O.pdhg(pb, 8000)
    m = (1 - gamma * xi[0] ** 2, -gamma * xi[0] * xi[1], 1 - gamma * xi[1] ** 2)
    ref = _fista_rof_dual(f, 0.15, 60000, pointwise_mat=m)
    np.testing.assert_allclose(res.u, ref, atol=5e-6)
    # gamma = 0 reduces directional TV to TV, iterate for iterate
    pb0 = _denoise_problem(f, O.REG_DTV, 0.15, xi=xi, gamma=0.0)
    pbt = _denoise_problem(f, O.REG_TV, 0.15)
    np.testing.assert_array_equal(O.pdhg(pb0, 50).u, O.pdhg(pbt, 50).u)


def test_pdhg_tgv_denoise_matches_admm():
    rng = np.random.default_rng(7)
    n = 5
    iy, ix = np.mgrid[0:n, 0:n] / n
    f = 0.8 * ix + 0.3 * iy + (ix > 0.5) + 0.05 * rng.standard_normal((n, n))
    alpha, beta = 0.1, 2.0
    pb = _denoise_problem(f, O.REG_TGV, alpha, beta=beta)
    res = O.pdhg(pb, 20000)
    ref = _admm_tgv_denoise(f, alpha, beta, 20000)
    np.testing.assert_allclose(res.u, ref, atol=1e-5)


def test_pdhg_tgv_denoise_beta_large_is_tv_like_limit():
    """beta -> infinity forces E v = 0, i.e. v = 0 here, so TGV reduces to TV."""
    rng = np.random.default_rng(8)
    n = 5
    f = (rng.uniform(size=(n, n)) > 0.5) + 0.1 * rng.standard_normal((n, n))
    tgv = O.pdhg(_denoise_problem(f, O.REG_TGV, 0.12, beta=1e6), 20000)
    ref = _fista_rof_dual(f, 0.12, 40000)
    np.testing.assert_allclose(tgv.u, ref, atol=1e-4)


@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV])
def test_large_alpha_gives_constant_fit(reg):
    """alpha -> infinity: the solution lies in the regulariser's null space (constants
    under the Neumann / -(d^+)^T discretisation) and fits the data there:
    u = c 1 with c = <K1, f>/||K1||^2."""
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    f = np.random.default_rng(reg).uniform(0.0, 1.0, Km.shape[0])
    pb = O.problem_from_matrix(Km, g.n, f, reg=reg, alpha=1e3, beta=1.0)
    res = O.pdhg(pb, 20000)
    k1 = Km @ np.ones(g.n * g.n)
    c = float(k1 @ f) / float(k1 @ k1)
    np.testing.assert_allclose(res.u, c, atol=1e-5)


def test_zero_alpha_gives_least_squares():
    rng = np.random.default_rng(11)
    n = 3
    Km = rng.uniform(0.0, 1.0, (30, n * n))
    u_true = rng.standard_normal(n * n)
    f = Km @ u_true + 0.01 * rng.standard_normal(30)
    pb = O.problem_from_matrix(Km, n, f, reg=O.REG_TV, alpha=0.0)
    res = O.pdhg(pb, 60000)
    ls = np.linalg.lstsq(Km, f, rcond=None)[0]
    np.testing.assert_allclose(res.u.ravel(), ls, atol=1e-6)


# ---------------------------------------------------------------------------
# step sizes
# ---------------------------------------------------------------------------

def _stacked_A(pb, Km):
    B = O.regulariser_operator(pb)
    nx = B.shape[1]
    Kx = sp.hstack([Km, sp.csr_matrix((Km.shape[0], nx - Km.shape[1]))]) if nx > Km.shape[1] else Km
    return sp.vstack([Kx, B]).toarray()


@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV, O.REG_DTV])
def test_diag_preconditioner_norm_bound(reg):
    g = _geom(n=5, n_det=3, n_t=6, m=16)
    Km = O.system_matrix(g)
    rng = np.random.default_rng(reg)
    xi = rng.standard_normal((2, 5, 5))
    xi /= np.sqrt(xi[0] ** 2 + xi[1] ** 2 + 0.2)
    pb = O.problem_from_matrix(Km, g.n, np.zeros(Km.shape[0]), reg=reg, xi=xi)
    st = O.diag_steps(pb)
    A = _stacked_A(pb, Km)
    sig = [st.sig_q, st.sig_r.ravel(), st.sig_r.ravel()]
    tau = [st.tau_u.ravel()]
    if reg == O.REG_TGV:
        sig += [st.sig_s.ravel()] * 3
        tau += [st.tau_v.ravel()]
    S = np.concatenate(sig)
    T = np.concatenate(tau)
    M = np.sqrt(S)[:, None] * A * np.sqrt(T)[None, :]
    assert np.linalg.norm(M, 2) <= 1 + 1e-9
    # the primal-dual balance leaves the norm unchanged
    for ratio in (0.1, 7.0):
        sb = O.balanced_steps(st, ratio)
        Sb = np.concatenate([sb.sig_q, sb.sig_r.ravel(), sb.sig_r.ravel()] +
                            ([sb.sig_s.ravel()] * 3 if reg == O.REG_TGV else []))
        Tb = np.concatenate([sb.tau_u.ravel()] + ([sb.tau_v.ravel()] if reg == O.REG_TGV else []))
        assert np.allclose(Sb * ratio, S) and np.allclose(Tb / ratio, T)
        Mb = np.sqrt(Sb)[:, None] * A * np.sqrt(Tb)[None, :]
        assert abs(np.linalg.norm(Mb, 2) - np.linalg.norm(M, 2)) < 1e-9
    # and it is the Pock-Chambolle choice: rows of |A| sum to 1/sigma where ungrouped
    np.testing.assert_allclose(np.abs(A[:Km.shape[0]]).sum(1)[Km.getnnz(1) > 0],
                               1 / st.sig_q[Km.getnnz(1) > 0], rtol=1e-12)
    np.testing.assert_allclose(np.abs(A).sum(0), 1 / T, rtol=1e-12)


@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV])
def test_scalar2_steps_bound(reg):
    g = _geom(n=5, n_det=3, n_t=6, m=16)
    Km = O.system_matrix(g)
    pb = O.problem_from_matrix(Km, g.n, np.zeros(Km.shape[0]), reg=reg)
    st = O.scalar2_steps(pb, power_iters=500)
    A = _stacked_A(pb, Km)
    L1 = np.linalg.norm(Km.toarray(), 2)
    B = O.regulariser_operator(pb).toarray()
    L2 = np.linalg.norm(B, 2)
    tau = st.tau_u.flat[0]
    assert math.sqrt(st.sig_q[0] * tau) * L1 + math.sqrt(st.sig_r.flat[0] * tau) * L2 < 1
    assert abs(1.0 / tau - L1) < 1e-6 * L1


# ---------------------------------------------------------------------------
# duality gap
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV, O.REG_DTV])
def test_gap_weak_duality_on_random_feasible_pairs(reg):
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    rng = np.random.default_rng(20 + reg)
    n = g.n
    xi = rng.standard_normal((2, n, n))
    xi /= np.sqrt(xi[0] ** 2 + xi[1] ** 2 + 0.2)
    f = rng.uniform(0, 2, Km.shape[0])
    pb = O.problem_from_matrix(Km, n, f, reg=reg, alpha=0.3, beta=0.5, xi=xi)
    for _ in range(20):
        u = rng.uniform(-pb.box_u, pb.box_u, (n, n))
        v = rng.uniform(-pb.box_v, pb.box_v, (2, n, n)) if reg == O.REG_TGV else None
        q = rng.standard_normal(Km.shape[0])
        r = O.proj_ball(rng.standard_normal((2, n, n)), pb.alpha)
        s = O.proj_ball(rng.standard_normal((3, n, n)), pb.alpha * pb.beta) if reg == O.REG_TGV else None
        assert O.duality_gap(pb, u, q, r, v, s)["gap"] >= -1e-10


@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV, O.REG_DTV])
def test_gap_stationarity_split_is_the_fenchel_young_identity(reg):
    """gap - stationarity must equal the Fenchel-Young gap F(Ax) + F*(y) - <Ax, y> of the
    dual variables, written here from F and A directly (the identity needs
    <Ax, y> = <x, A^T y>, so a wrong adjoint or sign fails it)."""
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    rng = np.random.default_rng(40 + reg)
    n = g.n
    xi = rng.standard_normal((2, n, n))
    xi /= np.sqrt(xi[0] ** 2 + xi[1] ** 2 + 0.2)
    f = rng.uniform(0, 2, Km.shape[0])
    pb = O.problem_from_matrix(Km, n, f, reg=reg, alpha=0.3, beta=0.5, xi=xi)
    for _ in range(5):
        u = rng.uniform(-1, 1, (n, n))
        v = rng.uniform(-1, 1, (2, n, n)) if reg == O.REG_TGV else None
        q = rng.standard_normal(Km.shape[0])
        r = O.proj_ball(rng.standard_normal((2, n, n)), pb.alpha)
        s = O.proj_ball(rng.standard_normal((3, n, n)), pb.alpha * pb.beta) if reg == O.REG_TGV else None
        gp = O.duality_gap(pb, u, q, r, v, s)
        Ku = Km @ u.ravel()
        fy = 0.5 * np.sum((Ku - f) ** 2) + 0.5 * q @ q + q @ f - Ku @ q
        gu = O.grad(u) if reg != O.REG_DTV else O.dtv_apply(xi, pb.gamma, O.grad(u))
        if reg == O.REG_TGV:
            gu = gu - v
        nrm = lambda p: np.sum(np.sqrt(np.sum(p * p, axis=0)))
        fy += pb.alpha * nrm(gu) - np.sum(gu * r)
        if reg == O.REG_TGV:
            e = O.sym_grad(v)
            fy += pb.alpha * pb.beta * nrm(e) - np.sum(e * s)
        assert fy >= -1e-10
        assert abs((gp["gap"] - gp["stationarity"]) - fy) < 1e-9 * (1 + abs(fy))


def test_cone_distance_against_brute_force():
    rng = np.random.default_rng(50)
    lam = np.linspace(0.0, 20.0, 200001)
    for _ in range(20):
        g = rng.standard_normal(3)
        p = rng.standard_normal(3)
        p *= 0.7 / np.linalg.norm(p)
        inside = O.pat_oracle._cone_distance(g[:, None, None], 0.5 * p[:, None, None], 0.7)[0, 0]
        assert abs(inside - np.linalg.norm(g)) < 1e-12          # interior: the cone is {0}
        on = O.pat_oracle._cone_distance(g[:, None, None], p[:, None, None], 0.7)[0, 0]
        brute = np.min(np.linalg.norm(g[:, None] - lam[None, :] * p[:, None] / 0.7, axis=0))
        assert abs(on - brute) < 1e-6


def test_pd_residuals_vanish_at_the_solution():
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    f = Km @ np.random.default_rng(3).uniform(0, 1, g.n * g.n)
    for reg in (O.REG_TV, O.REG_TGV):
        pb = O.problem_from_matrix(Km, g.n, f, reg=reg, alpha=0.05, beta=1.0)
        z = np.zeros((g.n, g.n))
        p0, d0 = O.pd_residuals(pb, z, np.zeros(f.size), np.zeros((2, g.n, g.n)),
                                np.zeros((2, g.n, g.n)), np.zeros((3, g.n, g.n)))
        res = O.pdhg(pb, 40000, tol=1e-9, gap_every=10, step_ratio=0.3 if reg == O.REG_TGV else 1.0)
        p1, d1 = O.pd_residuals(pb, res.u, res.q, res.r, res.v, res.s)
        assert p1 < 1e-3 * max(p0, d0) and d1 < 1e-3 * max(p0, d0)


def test_adaptive_balance_rule_and_convergence():
    # the rule: no move inside the dead zone, sqrt of the ratio clamped to [1/2, 2]
    assert O.balance_update(3.0, 1.0, 1.5, 0) == (3.0, 0)          # ratio 1/1.5: inside
    s1, k = O.balance_update(1.0, 9.0, 1.0, 0)                       # ratio 9: factor 2 (clamped)
    assert (s1, k) == (2.0, 1)
    s2, k = O.balance_update(1.0, 1.0, 4.0, 4)                       # ratio 1/4: factor 1/2, decayed
    assert abs(s2 - 0.5 ** (0.97 ** 4)) < 1e-15 and k == 5
    # an adaptive run reaches the same saddle point as a fixed one
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    f = Km @ np.random.default_rng(2).uniform(0, 1, g.n * g.n)
    pb = O.problem_from_matrix(Km, g.n, f, reg=O.REG_TGV, alpha=0.05, beta=1.0)
    a = O.pdhg(pb, 20000, tol=1e-6, gap_every=10, adapt=True)
    b = O.pdhg(pb, 20000, tol=1e-6, gap_every=10)
    assert a.gap["rel_gap"] <= 1e-6 and b.gap["rel_gap"] <= 1e-6
    assert a.step_ratio != 1.0
    assert np.linalg.norm(a.u - b.u) <= 1e-3 * np.linalg.norm(b.u)


def test_gap_zero_at_known_saddle_point_and_decays():
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    n = g.n
    pb = O.problem_from_matrix(Km, n, np.zeros(Km.shape[0]), reg=O.REG_TGV)
    z = np.zeros((n, n))
    gp = O.duality_gap(pb, z, np.zeros(Km.shape[0]), np.zeros((2, n, n)), np.zeros((2, n, n)),
                       np.zeros((3, n, n)))
    assert gp["gap"] == 0.0
    f = Km @ np.random.default_rng(0).uniform(0, 1, n * n)
    pb = O.problem_from_matrix(Km, n, f, reg=O.REG_TV, alpha=0.05)
    res = O.pdhg(pb, 3000, gap_every=100)
    gaps = [h[2] for h in res.history]
    assert gaps[-1] < 1e-6
    assert gaps[-1] < gaps[0]


def test_pdhg_tolerance_stop_and_warm_start_resume():
    g = _geom(n=6, n_det=3, n_t=8, m=24)
    Km = O.system_matrix(g)
    f = Km @ np.random.default_rng(1).uniform(0, 1, g.n * g.n)
    pb = O.problem_from_matrix(Km, g.n, f, reg=O.REG_TGV, alpha=0.05, beta=1.0)
    res = O.pdhg(pb, 5000, tol=1e-3, gap_every=10)
    assert res.iters_done < 5000 and res.iters_done % 10 == 0
    assert res.gap["rel_gap"] <= 1e-3
    # splitting a run in two with the warm-start entry gives the same iterates when the
    # extrapolated point equals the iterate (theta = 0)
    a = O.pdhg(pb, 40, theta=0.0)
    b1 = O.pdhg(pb, 25, theta=0.0)
    b2 = O.pdhg(pb, 15, theta=0.0, x0={"u": b1.u, "v": b1.v}, y0={"q": b1.q, "r": b1.r, "s": b1.s})
    np.testing.assert_allclose(b2.u, a.u, atol=1e-13)


# ---------------------------------------------------------------------------
# residual (reading R8) and the dTV direction field (reading R9)
# ---------------------------------------------------------------------------

def test_residual_hand_computed_two_step_sequence():
    """||x^{n+1} - x^n|| / ||x^n|| on a hand-worked sequence x^0 -> x^1 -> x^2 of a primal
    pair (u, v); the numbers are chosen so that dividing by ||x^{n+1}|| (or by the squared
    norm, or dropping v) gives a different value."""
    u0 = np.array([[2.0, 0.0], [1.0, 2.0]])            # |u0| = 3
    v0 = np.zeros((2, 2, 2))
    v0[1, 0, 1] = 4.0                                   # |x^0| = 5
    u1 = u0.copy()
    u1[1, 1] += 3.0                                     # step (3, 4): |x^1 - x^0| = 5
    v1 = v0.copy()
    v1[0, 1, 0] = 4.0                                   # |x^1|^2 = 4+1+25+16+16 = 62
    assert O.residual([u1, v1], [u0, v0]) == pytest.approx(5.0 / 5.0, rel=1e-15)
    u2 = u1.copy()
    u2[0, 1] = 6.0                                      # step (6, 0): |x^2 - x^1| = 6
    assert O.residual([u2, v1], [u1, v1]) == pytest.approx(6.0 / math.sqrt(62.0), rel=1e-15)
    # the wrong denominator |x^{n+1}| = sqrt(98) would give 6 / 9.899, not 6 / 7.874
    assert abs(O.residual([u2, v1], [u1, v1]) - 6.0 / math.sqrt(98.0)) > 0.1
    # order matters: the old iterate is the second argument
    assert abs(O.residual([u1, v1], [u2, v1]) - O.residual([u2, v1], [u1, v1])) > 0.1
    # zero old iterate: 0 / 0 is 0, a step away from 0 is infinite
    z = np.zeros((2, 2))
    assert O.residual([z], [z]) == 0.0
    assert O.residual([u0], [z]) == math.inf


@pytest.mark.parametrize("reg", [O.REG_TV, O.REG_TGV])
def test_pdhg_residual_history_against_consecutive_runs(reg):
    """The residual the PDHG loop records after iteration n equals ||x^n - x^{n-1}|| /
    ||x^{n-1}|| computed from two independent runs of n-1 and n iterations."""
    rng = np.random.default_rng(11 + reg)
    n = 6
    Km = sp.csr_matrix(rng.uniform(0.0, 1.0, (20, n * n)) * (rng.uniform(size=(20, n * n)) < 0.3))
    f = Km @ rng.uniform(0.0, 1.0, n * n)
    pb = O.problem_from_matrix(Km, n, f, reg=reg, alpha=0.05, beta=1.0)
    k = 7
    res = O.pdhg(pb, k, gap_every=1)
    prev = O.pdhg(pb, k - 1, gap_every=0, final_gap=False)
    cur = O.pdhg(pb, k, gap_every=0, final_gap=False)
    xo = [prev.u] + ([prev.v] if reg == O.REG_TGV else [])
    xn = [cur.u] + ([cur.v] if reg == O.REG_TGV else [])
    num = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(xn, xo)))
    den = math.sqrt(sum(float(np.sum(b * b)) for b in xo))
    assert res.history[-1][0] == k
    assert res.history[-1][3] == pytest.approx(num / den, rel=1e-12)
    assert res.residual == pytest.approx(num / den, rel=1e-12)


def test_direction_field_of_a_ramp():
    """w = a ix + b iy has forward differences (a, b) inside the grid and zero difference
    across the last column / row (reading R2), so xi = (a, b) / sqrt(a^2 + b^2 + eta^2)
    inside, (0, b) / sqrt(b^2 + eta^2) on the last column, (a, 0) / sqrt(a^2 + eta^2) on
    the last row and 0 at the last pixel.  eta = 0.5 separates eta from eta^2."""
    n, a, b, eta = 7, -0.3, 0.4, 0.5
    iy, ix = np.mgrid[0:n, 0:n].astype(np.float64)
    w = a * ix + b * iy
    xi = O.direction_field(w, eta)
    assert xi.shape == (2, n, n)
    inner = np.array([a, b]) / math.sqrt(a * a + b * b + eta * eta)     # (-0.4243, 0.5657)
    np.testing.assert_allclose(xi[:, :-1, :-1], np.broadcast_to(inner[:, None, None], (2, n - 1, n - 1)),
                               rtol=0, atol=1e-15)
    np.testing.assert_allclose(xi[0, :-1, -1], 0.0, atol=0)
    np.testing.assert_allclose(xi[1, :-1, -1], b / math.sqrt(b * b + eta * eta), rtol=1e-15)
    np.testing.assert_allclose(xi[0, -1, :-1], a / math.sqrt(a * a + eta * eta), rtol=1e-15)
    np.testing.assert_allclose(xi[1, -1, :-1], 0.0, atol=0)
    assert xi[0, -1, -1] == 0.0 and xi[1, -1, -1] == 0.0
    # eta (not squared) would give |xi| = 0.5 / sqrt(0.75) = 0.577 instead of 0.707
    assert np.hypot(xi[0, 0, 0], xi[1, 0, 0]) == pytest.approx(math.sqrt(0.5), rel=1e-15)
    # the sign follows the gradient, and the field scales out: xi(c w, c eta) = xi(w, eta)
    np.testing.assert_allclose(O.direction_field(-3.0 * w, 3.0 * eta), -xi, rtol=1e-14, atol=1e-16)


def test_direction_field_limits():
    """|xi| < 1 everywhere, |xi| -> 1 where grad w != 0 as eta -> 0, and xi -> grad w / eta
    as eta -> infinity (the first-order term of 1/sqrt(g^2 + eta^2))."""
    rng = np.random.default_rng(5)
    w = rng.standard_normal((9, 9))
    xi = O.direction_field(w, 0.2)
    assert np.all(np.hypot(xi[0], xi[1]) < 1.0)
    gx = np.zeros_like(w)
    gx[:, :-1] = w[:, 1:] - w[:, :-1]
    gy = np.zeros_like(w)
    gy[:-1, :] = w[1:, :] - w[:-1, :]
    g = np.hypot(gx, gy)
    xi0 = O.direction_field(w, 1e-12)
    np.testing.assert_allclose(np.hypot(xi0[0], xi0[1])[g > 0], 1.0, rtol=1e-12)
    big = 1e6
    xib = O.direction_field(w, big)
    np.testing.assert_allclose(xib[0] * big, gx, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(xib[1] * big, gy, rtol=1e-10, atol=1e-12)
