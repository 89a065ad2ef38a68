"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, a textbook/library solution, an
exhaustive enumeration, an inequality of the paper, or a hand-derived value, chosen so
that a dropped term, a wrong sign, a wrong index or a transposed operand fails.
"""

import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O
from inputs import dc_problem, nesterov_lasso, random_lasso, ncquad_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(A, b, lam, **kw):
    return O.Problem(A=np.asarray(A, float), b=np.asarray(b, float), lam=lam, **kw)


# ---------------------------------------------------------------- soft threshold

def test_soft_threshold_hand_values():
    # Hand-computed values of sign(v) max(|v| - t, 0), including the tie |v| = t.
    with open(os.path.join(GOLDEN, "soft_threshold.json")) as f:
        cases = json.load(f)["cases"]
    for v, t, want in cases:
        assert O.soft(v, t) == want


# ---------------------------------------------------------------- orthogonal designs

def test_diagonal_design_closed_form():
    """A = diag(s): min 0.5 (s_j x_j - b_j)^2 + lam |x_j| has x_j = soft(s_j b_j, lam) / s_j^2."""
    rng = np.random.default_rng(1)
    n = 9
    s = rng.uniform(0.5, 3.0, n) * rng.choice([-1, 1], n)
    b = rng.standard_normal(n) * 2
    lam = 0.7
    want = np.sign(s * b) * np.maximum(np.abs(s * b) - lam, 0) / s ** 2
    p = _prob(np.diag(s), b, lam)
    d = O.surrogate_weights(p)
    # One Jacobi sweep with gamma = 1 from any start is exact for a diagonal Gram matrix.
    x0 = rng.standard_normal(n)
    x, _ = O.jacobi_sweep(p, x0, O.residual(p, x0), d, 1.0)
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-14)
    # Same for Gauss-Seidel with blocks of 4.
    x2, _ = O.gauss_seidel_sweep(p, x0, O.residual(p, x0), d, 1.0, w=4)
    np.testing.assert_allclose(x2, want, rtol=0, atol=1e-14)


def test_identity_design_with_box_closed_form():
    """A = I with box [lo, hi]: the separable minimiser is clip(soft(b, lam), lo, hi)."""
    rng = np.random.default_rng(2)
    n = 12
    b = rng.standard_normal(n) * 3
    lo = -rng.uniform(0.1, 2, n)
    hi = rng.uniform(0.1, 2, n)
    lo[0], hi[0] = 0.5, 1.5       # box excluding 0
    lo[1], hi[1] = -1.5, -0.25
    lam = 0.8
    want = np.clip(np.sign(b) * np.maximum(np.abs(b) - lam, 0), lo, hi)
    p = _prob(np.eye(n), b, lam, lo=lo, hi=hi)
    x, _ = O.jacobi_sweep(p, np.zeros(n), O.residual(p, np.zeros(n)), O.surrogate_weights(p), 1.0)
    np.testing.assert_allclose(x, want, atol=1e-15)


# ---------------------------------------------------------------- best response

@pytest.mark.parametrize("seed", range(6))
def test_best_response_matches_grid_minimisation(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        x = rng.standard_normal() * 2
        g = rng.standard_normal() * 3
        d = rng.uniform(0.1, 4)
        lam = rng.uniform(0, 2)
        lo, hi = sorted(rng.uniform(-3, 3, 2))
        if rng.random() < 0.3:
            lo, hi = -np.inf, np.inf
        phi = lambda y: g * (y - x) + 0.5 * d * (y - x) ** 2 + lam * np.abs(y)  # noqa: E731
        a = max(lo, -20.0)
        b = min(hi, 20.0)
        grid = np.linspace(a, b, 400001)
        ybest = grid[np.argmin(phi(grid))]
        got = float(O.best_response(x, g, d, lam, lo, hi))
        assert abs(got - ybest) <= 2 * (b - a) / 400000
        assert phi(got) <= phi(ybest) + 1e-12


def test_best_response_zero_weight_rule():
    # d = 0 (a zero column without proximal term) -> clip(0, lo, hi)
    assert O.best_response(1.0, 0.0, 0.0, 1.0, -1, 1) == 0.0
    assert O.best_response(1.0, 0.0, 0.0, 1.0, 0.5, 1) == 0.5


# ---------------------------------------------------------------- whole-solver pins

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gs_limit_equals_brute_force_lasso(seed):
    d = random_lasso(30, 7, seed=seed, lam=0.9)
    p = O.Problem.from_data(d)
    sols = O.brute_force_lasso(p.A, p.b, p.lam)
    assert len(sols) == 1
    x, F, _ = O.solve_gs(p, gamma=1.0, w=1, max_sweeps=5000, tol=1e-15)
    np.testing.assert_allclose(x, sols[0], atol=1e-8)
    assert O.kkt_violation(p, sols[0]) < 1e-10


def test_gs_limit_matches_scipy_bound_constrained_qp():
    """LASSO as a smooth bound-constrained problem in (u, v) >= 0, x = u - v (L-BFGS-B)."""
    d = random_lasso(40, 12, seed=5, lam=0.5)
    p = O.Problem.from_data(d)
    A, b, lam = p.A, p.b, p.lam
    n = p.n

    def fun(z):
        x = z[:n] - z[n:]
        r = A @ x - b
        g = A.T @ r
        return 0.5 * r @ r + lam * z.sum(), np.concatenate([g + lam, -g + lam])

    res = minimize(fun, np.zeros(2 * n), jac=True, method="L-BFGS-B",
                   bounds=[(0, None)] * (2 * n), options=dict(ftol=1e-15, gtol=1e-12, maxiter=20000))
    x_ref = res.x[:n] - res.x[n:]
    x, F, _ = O.solve_gs(p, gamma=0.9, w=3, max_sweeps=20000, tol=1e-15)
    np.testing.assert_allclose(x, x_ref, atol=1e-6)
    assert abs(F - res.fun) <= 1e-9 * abs(res.fun)


def test_least_squares_special_case():
    """lam = 0, no box, full column rank: the limit is the least-squares solution."""
    d = random_lasso(50, 10, seed=3, lam=0.0)
    p = O.Problem.from_data(d)
    x_ls = np.linalg.lstsq(p.A, p.b, rcond=None)[0]
    x, _, _ = O.solve_gs(p, gamma=1.0, w=2, max_sweeps=20000, tol=1e-16)
    np.testing.assert_allclose(x, x_ls, atol=1e-9)


def test_planted_nesterov_optimum():
    d = nesterov_lasso(60, 200, 10, lam=1.0, seed=0)
    p = O.Problem.from_data(d)
    xs = d["x_star"]
    # generator: residual at x* is -y*, so F(x*) equals the closed form
    np.testing.assert_allclose(O.residual(p, xs), -d["y_star"], atol=1e-12)
    assert abs(O.objective(p, xs) - d["f_star"]) <= 1e-12 * d["f_star"]
    assert O.kkt_violation(p, xs) < 1e-11
    # GS from 0 reaches the planted optimum
    x, F, _ = O.solve_gs(p, gamma=0.9, w=1, max_sweeps=20000, tol=1e-16)
    assert (F - d["f_star"]) / d["f_star"] < 1e-12
    np.testing.assert_allclose(x, xs, atol=1e-7)


def test_planted_optimum_fp32_storage_gap_is_tiny():
    """With FP32 storage the planted x* stays optimal up to ~1e-10 relative in F."""
    d = nesterov_lasso(80, 300, 12, lam=1.0, seed=4, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    x, F, _ = O.solve_gs(p, x0=d["x_star"], gamma=1.0, w=1, max_sweeps=2000, tol=1e-16)
    F_xs = O.objective(p, d["x_star"])
    assert F <= F_xs + 1e-12 * F_xs
    assert (F_xs - F) / F < 1e-9
    assert abs(F_xs - d["f_star"]) / d["f_star"] < 1e-6


# ---------------------------------------------------------------- paper inequalities

@pytest.mark.parametrize("loss", ["lasso", "ncquad"])
def test_proposition1_descent_inequality(loss):
    """(x^_i - y_i)^T grad_i f(y) + g_i(x^_i) - g_i(y_i) <= -c ||x^_i - y_i||^2 (Prop. 1)."""
    rng = np.random.default_rng(7)
    if loss == "lasso":
        d = random_lasso(25, 16, seed=7, lam=0.4, box=1.0)
        p = O.Problem.from_data(d)
    else:
        d = ncquad_problem(40, 16, seed=7)
        p = O.Problem.from_data(d, loss="ncquad")
    dw = O.surrogate_weights(p, tau=0.3)
    lo, hi = p.lo_or_inf(), p.hi_or_inf()
    for _ in range(50):
        y = np.clip(rng.standard_normal(p.n), lo, hi)
        g = O.gradient(p, y)
        for cols in O.block_ranges(p.n, 4):
            xh = O.best_response(y[cols], g[cols], dw[cols], p.lam, lo[cols], hi[cols])
            lhs = (xh - y[cols]) @ g[cols] + p.lam * (np.abs(xh).sum() - np.abs(y[cols]).sum())
            c = dw[cols].min()
            assert lhs <= -c * np.sum((xh - y[cols]) ** 2) + 1e-10


def test_sequential_descent_bound():
    """Delay 0: F(x+) <= F(x) - gamma (d_j - gamma kappa_j / 2) |x^_j - x_j|^2 per update."""
    d = random_lasso(30, 20, seed=8, lam=0.3)
    p = O.Problem.from_data(d)
    kap = O.coord_curvature(p)
    dw = O.surrogate_weights(p, tau=0.1)
    x = np.zeros(p.n)
    r = O.residual(p, x)
    gamma = 0.9
    for sweep in range(5):
        for j in range(p.n):
            F0 = O.objective(p, x)
            xn, r = O.gauss_seidel_sweep(p, x, r, dw, gamma, w=1, order=[j])
            step = (xn[j] - x[j]) / gamma
            F1 = O.objective(p, xn)
            assert F1 <= F0 - gamma * (dw[j] - gamma * kap[j] / 2) * step ** 2 + 1e-10
            x = xn


def test_jacobi_descends_with_safe_tau():
    d = random_lasso(40, 60, seed=9, lam=0.2)
    p = O.Problem.from_data(d)
    gamma = 0.9
    tr = O.jacobi_tau_rel(p, gamma)
    dw = O.surrogate_weights(p, tau_rel=tr)
    x = np.zeros(p.n)
    r = O.residual(p, x)
    F = O.objective(p, x)
    for _ in range(40):
        x, r = O.jacobi_sweep(p, x, r, dw, gamma)
        Fn = O.objective(p, x)
        assert Fn <= F + 1e-12
        F = Fn


def test_coordinate_descent_is_exact_coordinate_minimisation():
    """w = 1, tau = 0, gamma = 1: after the update the coordinate satisfies its 1-D optimality."""
    d = random_lasso(20, 15, seed=10, lam=0.5)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(p.n)
    r = O.residual(p, x)
    for j in range(p.n):
        x, r = O.gauss_seidel_sweep(p, x, r, dw, 1.0, w=1, order=[j])
        gj = p.A[:, j] @ (p.A @ x - p.b)
        if x[j] == 0:
            assert abs(gj) <= p.lam + 1e-12
        else:
            assert abs(gj + p.lam * np.sign(x[j])) < 1e-12


@pytest.mark.parametrize("loss", ["lasso", "ncquad"])
def test_scalar_update_minimises_objective_along_coordinate(loss):
    """tau = 0, gamma = 1, w = 1: the surrogate is f restricted to x_j, so the update is
    the exact minimiser of F along coordinate j within the box (grid search of F)."""
    d = ncquad_problem(20, 8, seed=21, lam_frac=0.2)
    p = O.Problem.from_data(d, loss=loss)
    dw = O.surrogate_weights(p)
    assert np.all(dw > 0)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, p.n)
    r = O.residual(p, x)
    for j in range(p.n):
        x, r = O.gauss_seidel_sweep(p, x, r, dw, 1.0, w=1, order=[j])
        grid = np.linspace(-1, 1, 200001)
        vals = []
        for t in grid[::50]:
            z = x.copy()
            z[j] = t
            vals.append(O.objective(p, z))
        t0 = grid[::50][int(np.argmin(vals))]
        fine = np.linspace(max(-1, t0 - 1e-3), min(1, t0 + 1e-3), 2001)
        best = np.inf
        for t in fine:
            z = x.copy()
            z[j] = t
            best = min(best, O.objective(p, z))
        assert O.objective(p, x) <= best + 1e-10


def test_delay_zero_equals_gauss_seidel():
    d = random_lasso(25, 30, seed=11, lam=0.3)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=0.5)
    x0 = np.zeros(p.n)
    r0 = O.residual(p, x0)
    xa, _ = O.delayed_sweeps(p, x0, r0, dw, 0.8, 4, 0, 3, np.random.default_rng(0))
    xb, rb = x0, r0
    for _ in range(3):
        xb, rb = O.gauss_seidel_sweep(p, xb, rb, dw, 0.8, w=4)
    np.testing.assert_allclose(xa, xb, atol=1e-14)


def test_delayed_sweeps_use_stale_residual():
    """With a fixed delay of one update the result differs from GS but still converges."""
    d = random_lasso(30, 24, seed=12, lam=0.3)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=1.0)
    x_ref = O.brute_force_lasso(p.A[:, :8], p.b, p.lam)  # smoke of enumeration size
    assert len(x_ref) == 1
    x0 = np.zeros(p.n)
    xg, _ = O.gauss_seidel_sweep(p, x0, O.residual(p, x0), dw, 0.9, w=2)
    xd, _ = O.delayed_sweeps(p, x0, O.residual(p, x0), dw, 0.9, 2, 3, 1, np.random.default_rng(1))
    assert np.abs(xg - xd).max() > 1e-6
    xd, _ = O.delayed_sweeps(p, x0, O.residual(p, x0), dw, 0.9, 2, 3, 400, np.random.default_rng(1))
    xs, Fs, _ = O.solve_gs(p, gamma=1.0, max_sweeps=20000, tol=1e-16)
    assert abs(O.objective(p, xd) - Fs) <= 1e-9 * abs(Fs)


# ---------------------------------------------------------------- optimality measures

def test_gradient_matches_finite_differences():
    for loss in ("lasso", "ncquad"):
        d = ncquad_problem(30, 12, seed=13)
        p = O.Problem.from_data(d, loss=loss)
        x = np.random.default_rng(1).standard_normal(p.n)

        def fsmooth(z):
            r = p.A @ z - p.b
            return 0.5 * r @ r if loss == "lasso" else r @ r - p.c * z @ z

        h = 1e-6
        fd = np.array([(fsmooth(x + h * e) - fsmooth(x - h * e)) / (2 * h) for e in np.eye(p.n)])
        np.testing.assert_allclose(O.gradient(p, x), fd, rtol=1e-6, atol=1e-6)


def test_mf_zero_exactly_at_stationary_points_box():
    d = random_lasso(12, 5, seed=14, lam=0.3, box=0.6)
    p = O.Problem.from_data(d)
    pts = O.stationary_points_box(p)
    assert len(pts) == 1            # convex: unique
    assert O.stationarity(O.mf_measure(p, pts[0]), pts[0]) < 1e-10
    x, _, _ = O.solve_gs(p, gamma=1.0, max_sweeps=20000, tol=1e-16)
    np.testing.assert_allclose(x, pts[0], atol=1e-8)
    rng = np.random.default_rng(0)
    for _ in range(10):
        y = np.clip(rng.standard_normal(p.n), -0.6, 0.6)
        if np.abs(y - pts[0]).max() > 1e-3:
            assert O.stationarity(O.mf_measure(p, y), y) > 1e-6


def test_ncquad_limits_are_enumerated_stationary_points():
    d = ncquad_problem(6, 5, seed=15, lam_frac=0.05)
    p = O.Problem.from_data(d, loss="ncquad")
    kap = O.coord_curvature(p)
    assert np.all(kap > 0)
    pts = O.stationary_points_box(p)
    assert len(pts) >= 1
    for pt in pts:
        assert O.stationarity(O.mf_measure(p, pt), pt) < 1e-9
        assert O.stationarity(O.xhat_merit(p, pt, O.surrogate_weights(p)), pt) < 1e-9
    rng = np.random.default_rng(3)
    for trial in range(6):
        x0 = rng.uniform(-1, 1, p.n)
        x, F, _ = O.solve_gs(p, x0=x0, gamma=0.9, w=1, max_sweeps=50000, tol=1e-16)
        dist = min(np.abs(x - pt).max() for pt in pts)
        assert dist < 1e-6, (trial, x, pts)


def test_lambda_max_gram_matches_eigvalsh():
    d = random_lasso(30, 20, seed=16)
    p = O.Problem.from_data(d)
    kap = O.coord_curvature(p)
    M = (p.A / np.sqrt(kap)).T @ (p.A / np.sqrt(kap))
    want = np.linalg.eigvalsh(M).max()
    assert abs(O.lambda_max_gram(p.A, kap, iters=2000) - want) < 1e-8 * want


def test_linear_term_gradient_and_objective_by_finite_differences():
    d = ncquad_problem(25, 10, seed=18)
    for loss in ("lasso", "ncquad"):
        p = O.Problem.from_data(d, loss=loss)
        p.lin = np.random.default_rng(2).standard_normal(p.n)
        x = np.random.default_rng(3).standard_normal(p.n)
        lam = p.lam
        p.lam = 0.0                                  # smooth part only
        h = 1e-6
        fd = np.array([(O.objective(p, x + h * e) - O.objective(p, x - h * e)) / (2 * h) for e in np.eye(p.n)])
        np.testing.assert_allclose(O.gradient(p, x), fd, rtol=1e-6, atol=1e-6)
        p.lam = lam


def test_linear_term_solves_normal_equations():
    """lam = 0, b = 0, lin = -v: the minimiser of 0.5||Aw||^2 - v^T w solves A^T A w = v."""
    d = random_lasso(40, 9, seed=19, lam=0.0)
    p = O.Problem.from_data(d)
    p.b = np.zeros(p.m)
    v = np.random.default_rng(4).standard_normal(p.n)
    p.lin = -v
    w, _, _ = O.solve_gs(p, gamma=1.0, w=1, max_sweeps=50000, tol=1e-17)
    np.testing.assert_allclose(w, np.linalg.solve(p.A.T @ p.A, v), rtol=1e-8, atol=1e-9)


def test_adjoint_gradient_matches_finite_differences_of_exact_solutions():
    """dL/dlam and dL/db from the Cholesky adjoint against central differences (h = 1e-6) of
    exact LASSO minimisers (brute-force support enumeration), L = ||A_val x* - b_val||^2."""
    rng = np.random.default_rng(20)
    d = random_lasso(30, 8, seed=20, lam=0.4)
    A, b, lam = d["At"][:, :30].T.astype(np.float64), d["b"].astype(np.float64), d["lam"]
    Av = rng.standard_normal((12, 8))
    bv = rng.standard_normal(12)

    def solve(lam_, b_):
        sols = O.brute_force_lasso(A, b_, lam_)
        assert len(sols) == 1
        return sols[0]

    def loss(lam_, b_):
        x = solve(lam_, b_)
        r = Av @ x - bv
        return float(r @ r)

    x = solve(lam, b)
    assert 0 < np.count_nonzero(x) < 8
    v = 2.0 * Av.T @ (Av @ x - bv)
    dlam, db, _, S = O.lasso_adjoint_gradient(A, x, v)
    h = 1e-6
    fd_lam = (loss(lam + h, b) - loss(lam - h, b)) / (2 * h)
    assert abs(dlam - fd_lam) <= 1e-5 * max(1.0, abs(fd_lam))
    for i in range(0, 30, 7):
        e = np.zeros(30)
        e[i] = h
        fd_b = (loss(lam, b + e) - loss(lam, b - e)) / (2 * h)
        assert abs(db[i] - fd_b) <= 1e-5 * max(1.0, abs(fd_b))


def test_kkt_violation_detects_perturbation():
    d = nesterov_lasso(40, 100, 5, seed=17)
    p = O.Problem.from_data(d)
    xs = d["x_star"].copy()
    assert O.kkt_violation(p, xs) < 1e-11
    xs[d["support"][0]] *= 1.01
    assert O.kkt_violation(p, xs) > 1e-4


# ----------------------------------------------------------------- DC regularisers (Section 4.3)

@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
def test_dc_regulariser_definitions_and_split(reg):
    """h from its definition at points where it is known exactly; h- = eta|x| - h is convex,
    vanishes with its slope at 0, and its derivative is the central difference of
    eta|x| - h(x)."""
    theta = 20.0
    eta = O.dc_eta(reg, theta)
    assert eta == pytest.approx(theta if reg == "dc_exp" else theta / np.log(21.0), rel=1e-15)
    if reg == "dc_log":
        assert O.dc_h(reg, theta, 1.0) == pytest.approx(1.0, rel=1e-15)     # log(1+theta)/log(1+theta)
    else:
        assert O.dc_h(reg, theta, 1.0) == pytest.approx(1.0 - np.exp(-20.0), rel=1e-15)
    assert O.dc_h(reg, theta, 0.0) == 0.0
    assert O.dc_hminus_grad(reg, theta, 0.0) == 0.0
    hm = lambda t: eta * abs(t) - float(O.dc_h(reg, theta, t))
    for t in (-2.0, -0.3, -0.01, 0.004, 0.05, 0.7, 3.0):
        e = 1e-6 * max(1.0, abs(t))
        fd = (hm(t + e) - hm(t - e)) / (2 * e)
        assert float(O.dc_hminus_grad(reg, theta, t)) == pytest.approx(fd, rel=1e-6, abs=1e-7)
    grid = np.linspace(-2.0, 2.0, 4001)
    vals = eta * np.abs(grid) - O.dc_h(reg, theta, grid)
    assert np.all(vals[:-2] - 2 * vals[1:-1] + vals[2:] >= -1e-12)     # convex
    assert abs(hm(1e-5)) <= 1e-6                                       # h-(x) = o(x) at 0


@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
def test_dc_gauss_seidel_is_monotone(reg):
    """The coordinate surrogate keeps the quadratic exactly and linearises the concave
    -lam H- (an upper bound), so every best-response step lowers F (majorise-minimise)."""
    d = dc_problem(60, 120, reg=reg[3:], seed=3)
    p = O.Problem.from_data(d, loss=reg)
    dw = O.surrogate_weights(p)
    x, r = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    F = O.objective(p, x)
    for _ in range(20):
        x, r = O.gauss_seidel_sweep(p, x, r, dw, 1.0, w=1)
        Fn = O.objective(p, x)
        assert Fn <= F + 1e-12 * max(1.0, abs(F))
        F = Fn


@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
def test_dc_fixed_point_is_stationary_for_F(reg):
    """At a fixed point of the best-response map, F = ||Ax-b||^2 + lam H (evaluated from its
    definition) has zero partial derivatives on the support and non-negative one-sided
    directional derivatives off it (central / one-sided differences of F itself)."""
    d = dc_problem(50, 80, reg=reg[3:], seed=4)
    p = O.Problem.from_data(d, loss=reg)
    dw = O.surrogate_weights(p)
    x, r = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    for _ in range(3000):
        x, r = O.gauss_seidel_sweep(p, x, r, dw, 0.9, w=4)
    assert O.stationarity(O.xhat_merit(p, x, dw), x) < 1e-12
    assert 0 < np.count_nonzero(x) < p.n
    F = lambda y: O.objective(p, y)
    h = 1e-6
    for j in range(p.n):
        e = np.zeros(p.n)
        e[j] = h
        if x[j] != 0.0:
            assert abs((F(x + e) - F(x - e)) / (2 * h)) <= 1e-5
        else:
            assert (F(x + e) - F(x)) / h >= -1e-5
            assert (F(x - e) - F(x)) / h >= -1e-5


@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
def test_dc_coordinate_step_is_exact_minimisation_without_regulariser(reg):
    """With lam = 0 the DC loss is the plain quadratic ||Ax - b||^2; a unit step on one
    coordinate must land on the exact 1-D minimiser x_j - a_j^T r / ||a_j||^2 (pins the
    coordinate curvature 2||a_j||^2 of the surrogate)."""
    d = dc_problem(30, 12, reg=reg[3:], seed=5)
    p = O.Problem.from_data(d, loss=reg)
    p.lam = 0.0
    dw = O.surrogate_weights(p)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(p.n)
    r = O.residual(p, x)
    for j in range(p.n):
        xj, rj = O.gauss_seidel_sweep(p, x, r, dw, 1.0, w=1, order=[j])
        a = p.A[:, j]
        want = x[j] - float(a @ r) / float(a @ a)
        assert xj[j] == pytest.approx(want, rel=1e-12, abs=1e-12)


# ------------------------------------------------------------ diminishing stepsize (Section 4)

def test_diminishing_steps_recurrence_values():
    """gamma^{k+1} = gamma^k (1 - mu gamma^k): with gamma^0 = 1 and mu = 1/2 the sequence is
    exact in binary: 1, 1/2, 3/8, 39/128, ...; and 1/gamma^k - 1/gamma^0 lies between mu k and
    mu k + mu^2 sum_i gamma^i / (1 - mu gamma^i) (the recurrence of 1/gamma)."""
    g = O.diminishing_steps(1.0, 0.5, 4)
    assert list(g) == [1.0, 0.5, 0.375, 39.0 / 128.0]
    mu, K = 1e-3, 5000
    g = O.diminishing_steps(0.95, mu, K)
    assert np.all(np.diff(g) < 0) and g[-1] > 0
    inv = 1.0 / g - 1.0 / 0.95
    k = np.arange(K)
    assert np.all(inv >= mu * k - 1e-12)
    upper = mu * k + mu ** 2 * np.concatenate([[0.0], np.cumsum(g / (1 - mu * g))[:-1]])
    assert np.all(inv <= upper + 1e-9)


def test_gauss_seidel_with_step_sequence_equals_block_by_block_updates():
    """A sweep with a per-update step sequence applies steps[t] to its t-th update: the same
    as running the sweep one block at a time with that fixed step."""
    d = random_lasso(40, 24, seed=31, lam=0.1)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=0.1)
    steps = O.diminishing_steps(1.0, 0.05, 6)
    x0, r0 = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    xa, ra = O.gauss_seidel_sweep(p, x0, r0, dw, steps, w=4)
    xb, rb = x0, r0
    for t in range(6):
        xb, rb = O.gauss_seidel_sweep(p, xb, rb, dw, steps[t], w=4, order=[t])
    assert np.array_equal(xa, xb)


# ---------------------------------------------------------------- LASSO duality-gap certificate

def test_lasso_dual_gap_bounds_the_gap_and_vanishes_at_the_optimum():
    """Weak duality: P(x) - D(nu(x)) >= P(x) - F* >= 0 for any x, with F* from the exact
    enumeration; at the exact minimiser the certificate is ~0 (strong duality)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((14, 8))
    b = rng.standard_normal(14)
    lam = 0.6
    xs = O.brute_force_lasso(A, b, lam)
    assert len(xs) == 1
    p = O.Problem(A=A, b=b, lam=lam)
    Fstar = O.objective(p, xs[0])
    P, gap = O.lasso_dual_gap(p, xs[0])
    assert P == pytest.approx(Fstar, rel=1e-14) and abs(gap) <= 1e-10
    for _ in range(50):
        x = rng.standard_normal(8) * (rng.random(8) < 0.5)
        P, gap = O.lasso_dual_gap(p, x)
        assert gap >= P - Fstar - 1e-12 and P - Fstar >= -1e-12


def test_liu_wright_lambda_rule():
    from inputs import liu_wright_lasso
    d = liu_wright_lasso(200, 400, 5, sigma=0.01, seed=1)
    assert d["lam"] == pytest.approx(20 * np.sqrt(200 * np.log(400)) * 0.01, rel=1e-15)
    assert np.count_nonzero(d["xbar"]) == 5


# ---------------------------------------------------------------- block tables and orders

def test_block_steps_hand_table_ragged():
    """Jacobi step table (Algorithm 1 with the Section 4 stepsize rule, block i of a sweep
    takes steps[i]): n = 10 coordinates in blocks of w = 4 are {0..3}, {4..7}, {8, 9}."""
    got = O.block_steps(10, 4, [0.5, 0.25, 0.125])
    want = [0.5, 0.5, 0.5, 0.5, 0.25, 0.25, 0.25, 0.25, 0.125, 0.125]
    assert list(got) == want
    assert list(O.block_steps(3, 1, [1.0, 2.0, 3.0])) == [1.0, 2.0, 3.0]
    assert list(O.block_steps(5, 8, [0.75])) == [0.75] * 5


@pytest.mark.parametrize("w", [1, 3])
def test_random_sequential_visit_counts_on_a_diagonal_design(w):
    """Random-sequential order (the Corollary of Section 3: a uniformly drawn block, no delay)
    on A = diag(s), lam = 0.3: blocks decouple and the exact coordinate minimiser is
    x*_j = soft(s_j b_j, lam) / s_j^2, so a block visited k times with step gamma holds
    x* + (1 - gamma)^k (x0 - x*) and an unvisited block keeps x0.  The draws are over the
    ceil(n / w) blocks, reproduced here from the same seed."""
    n, gamma, count = 11, 0.6, 9
    rng = np.random.default_rng(3)
    s = rng.uniform(0.5, 2.0, n)
    b = rng.standard_normal(n) * 2
    lam = 0.3
    p = _prob(np.diag(s), b, lam)
    d = O.surrogate_weights(p)
    xstar = np.sign(s * b) * np.maximum(np.abs(s * b) - lam, 0) / s ** 2
    x0 = rng.standard_normal(n)
    x, r = O.random_sequential(p, x0, O.residual(p, x0), d, gamma, w, count, np.random.default_rng(17))
    nb = -(-n // w)
    draws = np.random.default_rng(17).integers(0, nb, size=count)
    visits = np.bincount(draws, minlength=nb)
    want = np.empty(n)
    for i in range(nb):
        cols = np.arange(i * w, min(n, (i + 1) * w))
        want[cols] = xstar[cols] + (1 - gamma) ** visits[i] * (x0[cols] - xstar[cols])
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r, s * x - b, rtol=0, atol=1e-13)
    # 9 draws: at w = 1 (11 blocks) some block stays unvisited, at w = 3 (4 blocks) some
    # block is visited more than once
    assert (visits == 0).any() if w == 1 else (visits > 1).any()


@pytest.mark.parametrize("gamma", [1.0, 0.7])
def test_solve_jacobi_is_damped_jacobi_for_the_normal_equations(gamma):
    """lam = 0, no box, d_j = ||a_j||^2: the Jacobi form of the block update is the textbook
    (damped) Jacobi iteration for A^T A x = A^T b, x_{k+1} = x_k - gamma D^{-1} A^T (A x_k - b),
    D = diag(A^T A); the residual it returns is A x - b."""
    rng = np.random.default_rng(8)
    m, n = 60, 12
    A = rng.standard_normal((m, n)) + 3.0 * np.eye(m, n) * 4
    b = rng.standard_normal(m)
    p = _prob(A, b, 0.0)
    d = O.surrogate_weights(p)
    x0 = rng.standard_normal(n)
    x, r = O.solve_jacobi(p, x0, d, gamma, 7)
    G = A.T @ A
    Dinv = 1.0 / np.diag(G)
    xr = x0.copy()
    for _ in range(7):
        xr = xr - gamma * Dinv * (G @ xr - A.T @ b)
    np.testing.assert_allclose(x, xr, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r, A @ x - b, rtol=1e-12, atol=1e-12)
