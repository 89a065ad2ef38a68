"""Plain FP64 reference implementation of the AsyFLEXA block update (numpy).

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

What is computed (Cannelli, Facchinei, Kungurtsev, Scutari, "Asynchronous Parallel
Algorithms for Nonconvex Big-Data Optimization, Part II"):

* Problem (eq. 1) specialised to  F(x) = f(x) + G(x),  G(x) = lam ||x||_1,
  X = box [lo, hi] (or R^n), no nonconvex constraints, with
    - LASSO (Section 4.2):              f(x) = 0.5 ||Ax - b||^2
    - nonconvex quadratic (Section 4.3): f(x) = ||Ax - b||^2 - c ||x||^2
  Writing r = Ax - b:  grad f = s A^T r - 2 c x  with s = 1 (LASSO) or 2, c = 0 (LASSO).
* Nonconvex sparse learning (Section 4.3): F(x) = ||Ax - b||^2 + lam H(x), H = sum_j h(x_j),
  with the exponential regulariser h(x) = 1 - exp(-theta |x|) or the logarithmic one
  h(x) = log(1 + theta |x|) / log(1 + theta).  Both are DC: h = h+ - h-, h+(x) = eta |x|,
  h-(x) = eta |x| - h(x) convex and smooth, eta = theta (exp) or theta / log(1 + theta) (log).
  The split used is f = ||Ax - b||^2 - lam H-(x) (smooth), G = lam eta ||x||_1: the
  printed assignment (f = h-, G = m + h+) would put the quadratic in G, which is not
  separable, so it is read as the one that fits Assumption A4.  The best response keeps the
  quadratic's exact coordinate curvature 2||a_j||^2, linearises -lam H- at the current point
  and keeps lam h+ (the subproblem of Section 4.3), i.e. the common closed form below with
  grad_j f = 2 a_j^T r - lam h-'(x_j) and l1 weight lam eta.

* Best response (eq. 2) with the surrogate of Section 4.2: for a scalar block the
  surrogate is f restricted to x_j plus (tau/2)(x_j - x~_j)^2, which for a quadratic f
  equals the linearisation plus (kappa_j + tau)/2 (x_j - x~_j)^2, kappa_j being the
  exact curvature of f along coordinate j (||a_j||^2 for LASSO, 2||a_j||^2 - 2c for the
  nonconvex quadratic).  Blocks of w > 1 coordinates use the same separable (diagonal)
  surrogate, so every coordinate's best response has the closed form
        x^_j = clip( soft(x~_j - grad_j / d_j,  lam / d_j),  lo_j, hi_j ),
  d_j = (1 + tau_rel) kappa_j + tau, soft(v, t) = sign(v) max(|v| - t, 0)
  (the soft-thresholding solution of Section 4; clipping after soft-thresholding is
  exact because the 1-D problem is convex).  d_j = 0 (a zero LASSO column with no
  proximal term) gives x^_j = clip(0, lo_j, hi_j).

* Fixed-step update (Algorithm 1, step S.4):  x_i <- x_i + gamma (x^_i(x~) - x_i).
  The experiments of Section 4 use the diminishing rule gamma^{k+1} = gamma^k (1 - mu gamma^k)
  instead, k counting updates; the sweep functions accept a per-update sequence of steps
  (``diminishing_steps``): update t of a Gauss-Seidel sweep uses steps[t], and in a Jacobi
  sweep block i uses steps[i].

* Execution orders (Algorithm 1 with different index/delay processes):
    - Jacobi: every block from the same x (the synchronous all-blocks form);
    - cyclic Gauss-Seidel: blocks 0..N-1 in order, each seeing all earlier updates
      (delay 0; used as the F* estimator of Section 4.2);
    - random sequential: uniformly drawn block, delay 0 (the Corollary of Section 3);
    - emulated delay: each update reads the residual of an earlier iterate x^{k-d},
      d <= delta drawn from a seeded generator (Assumption D1, inconsistent-read
      model of the Appendix), while the updated block itself is read current (D4).

* Optimality measures: M_F (Section 3, the argmin with unit weight), the merit
  ||x^(x) - x||_inf of Section 4.3, LASSO KKT residuals, F(x).

Everything here is FP64 and unoptimised.  Library primitives used: numpy matmul /
dot (for A^T r and A Delta) and numpy.linalg.solve (brute force).
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "soft", "residual", "objective", "gradient", "coord_curvature",
    "surrogate_weights", "best_response", "block_ranges", "jacobi_sweep",
    "gauss_seidel_sweep", "random_sequential", "delayed_sweeps", "mf_measure",
    "xhat_merit", "kkt_violation", "stationarity", "brute_force_lasso",
    "stationary_points_box", "lambda_max_gram", "jacobi_tau_rel", "solve_gs",
    "solve_jacobi", "lasso_support", "lasso_adjoint_gradient", "dc_eta", "dc_h", "dc_hminus_grad",
    "diminishing_steps", "block_steps", "lasso_dual_gap",
]

DC_LOSSES = ("dc_log", "dc_exp")


@dataclass
class Problem:
    """Problem data in FP64.  ``A`` is m x n (a view of the stored matrix)."""

    A: np.ndarray
    b: np.ndarray
    lam: float
    loss: str = "lasso"          # "lasso", "ncquad", "dc_log" or "dc_exp"
    c: float = 0.0
    theta: float = 0.0                 # regulariser parameter of the DC losses
    lo: np.ndarray | None = None
    hi: np.ndarray | None = None
    lin: np.ndarray | None = None      # optional linear term of f: f(x) += lin^T x
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]

    @property
    def s(self) -> float:
        """Factor of A^T r in grad f (1 for 0.5||Ax-b||^2, 2 for ||Ax-b||^2)."""
        return 1.0 if self.loss == "lasso" else 2.0

    @property
    def dc(self) -> bool:
        return self.loss in DC_LOSSES

    @property
    def l1(self) -> float:
        """Weight of ||x||_1 in G: lam, or lam * eta for the DC losses."""
        return self.lam * dc_eta(self.loss, self.theta) if self.dc else self.lam

    @staticmethod
    def from_data(d: dict, loss: str = "lasso", c: float | None = None, theta: float | None = None) -> "Problem":
        """Build from a generator dict (``At`` of shape (n, lda), column j = row j)."""
        m = d["m"]
        At = np.asarray(d["At"])[:, :m].astype(np.float64)
        lo = d.get("lo")
        hi = d.get("hi")
        return Problem(
            A=At.T, b=np.asarray(d["b"]).astype(np.float64), lam=float(d["lam"]),
            loss=loss, c=float(d.get("c", 0.0) if c is None else c),
            theta=float(d.get("theta", 0.0) if theta is None else theta),
            lo=None if lo is None else np.asarray(lo).astype(np.float64),
            hi=None if hi is None else np.asarray(hi).astype(np.float64),
            meta={k: v for k, v in d.items() if k not in ("At", "b", "lo", "hi")})

    def lo_or_inf(self) -> np.ndarray:
        return np.full(self.n, -np.inf) if self.lo is None else self.lo

    def hi_or_inf(self) -> np.ndarray:
        return np.full(self.n, np.inf) if self.hi is None else self.hi


# --------------------------------------------------------------------------- basics

def soft(v, t):
    """Soft-thresholding sign(v) * max(|v| - t, 0); exactly 0 when |v| <= t."""
    v = np.asarray(v, dtype=np.float64)
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def dc_eta(loss: str, theta: float) -> float:
    """eta(theta) of the DC split h = eta|x| - h- (Section 4.3)."""
    return float(theta) if loss == "dc_exp" else float(theta) / np.log1p(theta)


def dc_h(loss: str, theta: float, x) -> np.ndarray:
    """The regulariser h (Section 4.3), elementwise."""
    a = np.abs(np.asarray(x, dtype=np.float64))
    if loss == "dc_exp":
        return 1.0 - np.exp(-theta * a)
    return np.log1p(theta * a) / np.log1p(theta)


def dc_hminus_grad(loss: str, theta: float, x) -> np.ndarray:
    """Derivative of h-(x) = eta|x| - h(x): eta sign(x) - h'(x), which is 0 at x = 0."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    if loss == "dc_exp":
        return np.sign(x) * theta * (1.0 - np.exp(-theta * a))
    eta = dc_eta(loss, theta)
    return np.sign(x) * eta * (theta * a) / (1.0 + theta * a)


def residual(p: Problem, x: np.ndarray) -> np.ndarray:
    """r = A x - b."""
    return p.A @ x - p.b


def objective(p: Problem, x: np.ndarray) -> float:
    """F(x) = f(x) + lam ||x||_1 (eq. 1 with the Section 4 losses)."""
    r = residual(p, x)
    if p.dc:  # ||Ax - b||^2 + lam H(x)  (eq. of Section 4.3)
        F = float(r @ r) + p.lam * float(dc_h(p.loss, p.theta, x).sum())
        return F + (float(p.lin @ x) if p.lin is not None else 0.0)
    if p.loss == "lasso":
        f = 0.5 * float(r @ r)
    else:
        f = float(r @ r) - p.c * float(x @ x)
    if p.lin is not None:
        f += float(p.lin @ x)
    return f + p.lam * float(np.abs(x).sum())


def gradient(p: Problem, x: np.ndarray, r: np.ndarray | None = None) -> np.ndarray:
    """grad f(x) = s A^T r - 2 c x, with r = A x - b (recomputed if not given)."""
    if r is None:
        r = residual(p, x)
    g = p.s * (p.A.T @ r)
    if p.loss == "ncquad":
        g = g - 2.0 * p.c * x
    if p.dc:
        g = g - p.lam * dc_hminus_grad(p.loss, p.theta, x)
    if p.lin is not None:
        g = g + p.lin
    return g


def coord_curvature(p: Problem) -> np.ndarray:
    """kappa_j: second derivative of f along coordinate j."""
    sq = np.einsum("ij,ij->j", p.A, p.A)
    if p.loss == "lasso":
        return sq
    if p.dc:  # the quadratic part; the concave part is linearised in the surrogate
        return 2.0 * sq
    return 2.0 * sq - 2.0 * p.c


def surrogate_weights(p: Problem, tau: float = 0.0, tau_rel: float = 0.0) -> np.ndarray:
    """d_j = (1 + tau_rel) kappa_j + tau: curvature of the per-coordinate surrogate."""
    return (1.0 + tau_rel) * coord_curvature(p) + tau


def best_response(x, g, d, lam, lo, hi):
    """Closed-form minimiser of g (y - x) + d/2 (y - x)^2 + lam |y| over [lo, hi].

    Vectorised over coordinates; d <= 0 entries give clip(0, lo, hi).
    """
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    pos = d > 0
    dd = np.where(pos, d, 1.0)
    y = soft(x - g / dd, lam / dd)
    y = np.where(pos, y, 0.0)
    return np.minimum(np.maximum(y, lo), hi)


def diminishing_steps(gamma0: float, mu: float, count: int) -> np.ndarray:
    """gamma^0 = gamma0, gamma^{k+1} = gamma^k (1 - mu gamma^k): the stepsize sequence of the
    experiments of Section 4 (gamma^0 = 1, mu = 1e-6 there), for k = 0 .. count - 1."""
    g = np.empty(count)
    v = float(gamma0)
    for k in range(count):
        g[k] = v
        v = v * (1.0 - mu * v)
    return g


def block_steps(n: int, w: int, steps) -> np.ndarray:
    """Per-coordinate step for a Jacobi sweep where block i takes steps[i]."""
    out = np.empty(n)
    for i, cols in enumerate(block_ranges(n, w)):
        out[cols] = steps[i]
    return out


def block_ranges(n: int, w: int):
    """Blocks of w consecutive coordinates; the last block may be shorter."""
    return [np.arange(i, min(n, i + w)) for i in range(0, n, w)]


# ------------------------------------------------------------------ execution orders

def _block_step(p: Problem, x, r_tilde, d, gamma, cols, lo, hi):
    """One block update from residual r_tilde; returns Delta on ``cols`` (not applied)."""
    g = p.s * (p.A[:, cols].T @ r_tilde)
    if p.loss == "ncquad":
        g = g - 2.0 * p.c * x[cols]
    if p.dc:
        g = g - p.lam * dc_hminus_grad(p.loss, p.theta, x[cols])
    if p.lin is not None:
        g = g + p.lin[cols]
    xh = best_response(x[cols], g, d[cols], p.l1, lo[cols], hi[cols])
    return gamma * (xh - x[cols])


def jacobi_sweep(p: Problem, x, r, d, gamma):
    """All coordinates from the same (x, r); then x += Delta, r += A Delta."""
    lo, hi = p.lo_or_inf(), p.hi_or_inf()
    cols = np.arange(p.n)
    delta = _block_step(p, x, r, d, gamma, cols, lo, hi)
    x = x + delta
    nz = np.nonzero(delta)[0]
    r = r + p.A[:, nz] @ delta[nz]
    return x, r


def gauss_seidel_sweep(p: Problem, x, r, d, gamma, w=1, order=None):
    """Cyclic block Gauss-Seidel sweep: blocks in ``order`` (default 0..N-1).  ``gamma`` is a
    fixed step or a sequence with one step per update of the sweep (in update order)."""
    lo, hi = p.lo_or_inf(), p.hi_or_inf()
    blocks = block_ranges(p.n, w)
    x = x.copy()
    r = r.copy()
    seq = range(len(blocks)) if order is None else order
    per_update = np.ndim(gamma) > 0
    for t, i in enumerate(seq):
        cols = blocks[i]
        delta = _block_step(p, x, r, d, gamma[t] if per_update else gamma, cols, lo, hi)
        x[cols] += delta
        nz = np.nonzero(delta)[0]
        if nz.size:
            r += p.A[:, cols[nz]] @ delta[nz]
    return x, r


def random_sequential(p: Problem, x, r, d, gamma, w, n_updates, rng):
    """n_updates block updates, each on a uniformly drawn block, no delay."""
    nb = len(block_ranges(p.n, w))
    order = rng.integers(0, nb, size=n_updates)
    return gauss_seidel_sweep(p, x, r, d, gamma, w, order=order)


def delayed_sweeps(p: Problem, x, r, d, gamma, w, delta_max, sweeps, rng):
    """Cyclic sweeps where each update reads the residual of x^{k-d}, d <= delta_max.

    The updated block itself is read current (D4); every other coordinate is seen as
    in the stale iterate, i.e. the residual used is the one of the stale iterate with
    the current block substituted.
    """
    lo, hi = p.lo_or_inf(), p.hi_or_inf()
    blocks = block_ranges(p.n, w)
    x = x.copy()
    r = r.copy()
    hist_r = [r.copy()]
    hist_x = [x.copy()]
    for _ in range(sweeps):
        for cols in blocks:
            dly = int(rng.integers(0, min(delta_max, len(hist_r) - 1) + 1))
            r_old = hist_r[-1 - dly]
            x_old = hist_x[-1 - dly]
            # substitute the current value of the own block (D4)
            r_tilde = r_old + p.A[:, cols] @ (x[cols] - x_old[cols])
            step = _block_step(p, x, r_tilde, d, gamma, cols, lo, hi)
            x[cols] += step
            nz = np.nonzero(step)[0]
            if nz.size:
                r = r + p.A[:, cols[nz]] @ step[nz]
            hist_r.append(r.copy())
            hist_x.append(x.copy())
            if len(hist_r) > delta_max + 1:
                hist_r.pop(0)
                hist_x.pop(0)
    return x, r


def solve_gs(p: Problem, x0=None, d=None, gamma=1.0, w=1, max_sweeps=10000, tol=0.0):
    """Gauss-Seidel sweeps until F stops decreasing by more than tol (relative)."""
    x = np.zeros(p.n) if x0 is None else np.array(x0, dtype=np.float64)
    if d is None:
        d = surrogate_weights(p)
    r = residual(p, x)
    F = objective(p, x)
    for k in range(max_sweeps):
        x, r = gauss_seidel_sweep(p, x, r, d, gamma, w)
        r = residual(p, x)
        Fn = objective(p, x)
        if abs(F - Fn) <= tol * max(1.0, abs(Fn)):
            return x, Fn, k + 1
        F = Fn
    return x, F, max_sweeps


def solve_jacobi(p: Problem, x0, d, gamma, sweeps):
    """``sweeps`` Jacobi sweeps from x0 (incremental residual, as the method does)."""
    x = np.array(x0, dtype=np.float64)
    r = residual(p, x)
    for _ in range(sweeps):
        x, r = jacobi_sweep(p, x, r, d, gamma)
    return x, r


# -------------------------------------------------------------------- optimality

def mf_measure(p: Problem, x) -> np.ndarray:
    """M_F(x) = x - argmin_y { grad f(x)^T (y - x) + G(y) + 0.5||y - x||^2 } over X."""
    g = gradient(p, x)
    return x - best_response(x, g, np.ones(p.n), p.l1, p.lo_or_inf(), p.hi_or_inf())


def xhat_merit(p: Problem, x, d) -> np.ndarray:
    """x^(x) - x with the method's surrogate weights d (Section 4.3 merit)."""
    g = gradient(p, x)
    return best_response(x, g, d, p.l1, p.lo_or_inf(), p.hi_or_inf()) - x


def stationarity(v, x) -> float:
    """||v||_inf / max(1, ||x||_inf)."""
    return float(np.abs(v).max(initial=0.0) / max(1.0, float(np.abs(x).max(initial=0.0))))


def lasso_dual_gap(p: Problem, x) -> tuple[float, float]:
    """(P(x), P(x) - D(nu)) for the plain LASSO (no box, no linear term): nu = theta r with
    r = A x - b and theta = min(1, lam / ||A^T r||_inf) is feasible for the dual
    max -0.5||nu||^2 - b^T nu  s.t. ||A^T nu||_inf <= lam, so P(x) - D(nu) >= P(x) - F*
    (weak duality) bounds the optimality gap without knowing F*."""
    r = residual(p, x)
    P = 0.5 * float(r @ r) + p.lam * float(np.abs(x).sum())
    atr = float(np.abs(p.A.T @ r).max(initial=0.0))
    theta = 1.0 if atr <= p.lam else p.lam / atr
    D = -0.5 * theta * theta * float(r @ r) - theta * float(p.b @ r)
    return P, P - D


def kkt_violation(p: Problem, x) -> float:
    """LASSO optimality residual (no box): |g_j| <= lam off support, g_j = -lam sign(x_j) on it."""
    g = gradient(p, x)
    on = x != 0
    v_on = np.abs(g[on] + p.lam * np.sign(x[on]))
    v_off = np.maximum(np.abs(g[~on]) - p.lam, 0.0)
    return float(max(v_on.max(initial=0.0), v_off.max(initial=0.0)))


# ------------------------------------------------------------------- brute force

def brute_force_lasso(A, b, lam, tol=1e-9):
    """Exact LASSO minimiser for small n by enumerating sign patterns in {-1, 0, +1}^n.

    For a pattern sigma with support S the stationarity conditions on S read
    A_S^T (A_S x_S - b) = -lam sigma_S; the pattern is accepted when the solution has
    signs sigma_S and |a_j^T (A_S x_S - b)| <= lam off S.  Returns the accepted x
    (unique when A has full column rank).
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    found = []
    for sigma in itertools.product((-1, 0, 1), repeat=n):
        sig = np.array(sigma, dtype=np.float64)
        S = np.nonzero(sig)[0]
        x = np.zeros(n)
        if S.size:
            AS = A[:, S]
            rhs = AS.T @ b - lam * sig[S]
            try:
                xs = np.linalg.solve(AS.T @ AS, rhs)
            except np.linalg.LinAlgError:
                continue
            if np.any(np.sign(xs) != sig[S]):
                continue
            x[S] = xs
        r = A @ x - b
        off = np.setdiff1d(np.arange(n), S)
        if off.size and np.any(np.abs(A[:, off].T @ r) > lam * (1 + tol) + tol):
            continue
        found.append(x)
    return found


def stationary_points_box(p: Problem, tol=1e-9):
    """All stationary points of F over a box, by enumerating per-coordinate states.

    States: 'lo', 'hi' (at a bound), 'zero' (x_j = 0 strictly inside the box),
    'pos' / 'neg' (interior with fixed sign).  For free coordinates S the condition
    grad_S f = -lam sigma_S is linear (f is quadratic: grad f = H x - q with
    H = s A^T A - 2c I, q = s A^T b).  The candidate is kept when it satisfies every
    per-coordinate first-order condition 0 in grad_j f + lam d|x_j| + N_[lo_j,hi_j](x_j).
    Intended for n <= 6.
    """
    n = p.n
    lo, hi = p.lo_or_inf(), p.hi_or_inf()
    H = p.s * (p.A.T @ p.A) - 2.0 * p.c * np.eye(n)
    q = p.s * (p.A.T @ p.b)
    lam = p.lam
    pts = []
    for states in itertools.product(("lo", "hi", "zero", "pos", "neg"), repeat=n):
        x = np.zeros(n)
        free, sig = [], []
        ok = True
        for j, st in enumerate(states):
            if st == "lo":
                if not np.isfinite(lo[j]):
                    ok = False
                    break
                x[j] = lo[j]
            elif st == "hi":
                if not np.isfinite(hi[j]):
                    ok = False
                    break
                x[j] = hi[j]
            elif st == "zero":
                if not (lo[j] < 0.0 < hi[j]):
                    ok = False
                    break
            else:
                free.append(j)
                sig.append(1.0 if st == "pos" else -1.0)
        if not ok:
            continue
        free = np.array(free, dtype=np.int64)
        sig = np.array(sig)
        if free.size:
            fixed = np.setdiff1d(np.arange(n), free)
            rhs = q[free] - H[np.ix_(free, fixed)] @ x[fixed] - lam * sig
            try:
                x[free] = np.linalg.solve(H[np.ix_(free, free)], rhs)
            except np.linalg.LinAlgError:
                continue
        g = H @ x - q
        good = True
        for j, st in enumerate(states):
            if st == "pos":
                good = x[j] > max(lo[j], 0.0) + tol and x[j] < hi[j] - tol
            elif st == "neg":
                good = x[j] < min(hi[j], 0.0) - tol and x[j] > lo[j] + tol
            elif st == "zero":
                good = abs(g[j]) <= lam + tol
            elif st == "lo":
                # need some element of g_j + lam*d|lo| that is >= 0 (normal cone (-inf, 0])
                sub_hi = lam if lo[j] >= 0.0 else -lam
                good = g[j] + sub_hi >= -tol and lo[j] < hi[j]
            elif st == "hi":
                sub_lo = -lam if hi[j] <= 0.0 else lam
                good = g[j] + sub_lo <= tol and lo[j] < hi[j]
            if not good:
                break
        if good and not any(np.allclose(x, y, atol=1e-9, rtol=0) for y in pts):
            pts.append(x)
    return pts


# ------------------------------------------------------------- adjoint (not in the paper)

def lasso_support(x, rel_tol=1e-5):
    """Support of a LASSO solution: |x_j| > rel_tol * max(1, ||x||_inf)."""
    x = np.asarray(x, dtype=np.float64)
    return np.nonzero(np.abs(x) > rel_tol * max(1.0, float(np.abs(x).max(initial=0.0))))[0]


def lasso_adjoint_gradient(A, x, v, rel_tol=1e-5):
    """Gradient of L(x*(lam, b)) for the LASSO minimiser x* of 0.5||Ax - b||^2 + lam||x||_1.

    On the support S with signs s the optimality conditions A_S^T (A_S x_S - b) + lam s = 0
    are smooth in (lam, b); differentiating them gives dx_S = (A_S^T A_S)^-1 (A_S^T db - s dlam).
    With v = dL/dx* and w = (A_S^T A_S)^-1 v_S (FP64 Cholesky):
        dL/dlam = -s^T w,   dL/db = A_S w.
    Valid where the support and signs are locally constant.  Returns (dL/dlam, dL/db, w, S).
    """
    A = np.asarray(A, dtype=np.float64)
    S = lasso_support(x, rel_tol)
    s = np.sign(np.asarray(x, dtype=np.float64)[S])
    AS = A[:, S]
    G = AS.T @ AS
    L = np.linalg.cholesky(G)
    w = np.linalg.solve(L.T, np.linalg.solve(L, np.asarray(v, dtype=np.float64)[S]))
    return float(-(s @ w)), AS @ w, w, S


# ------------------------------------------------------------- parameter helpers

def lambda_max_gram(A, weights=None, iters=300, seed=0):
    """Largest eigenvalue of W^{-1/2} A^T A W^{-1/2} by power iteration (W = diag(weights))."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    w = np.ones(n) if weights is None else np.asarray(weights, dtype=np.float64)
    sc = np.where(w > 0, 1.0 / np.sqrt(np.where(w > 0, w, 1.0)), 0.0)
    v = np.random.default_rng(seed).standard_normal(n)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        u = sc * (A.T @ (A @ (sc * v)))
        lam = float(np.linalg.norm(u))
        if lam == 0.0:
            return 0.0
        v = u / lam
    return lam


def jacobi_tau_rel(p: Problem, gamma: float, margin: float = 1e-3, iters=300) -> float:
    """Smallest tau_rel (with tau = 0) for which a Jacobi sweep is a descent step.

    A Jacobi step decreases F whenever diag(d) - (gamma/2) Hess f is positive definite
    (sum the per-block inequality of Proposition 1 over all blocks and bound the
    quadratic remainder exactly, f being quadratic).  With d = (1 + tau_rel) kappa this
    holds when 1 + tau_rel > (gamma/2) lambda_max(K^-1/2 Hess K^-1/2).
    """
    kappa = coord_curvature(p)
    if p.loss == "lasso":
        lmax = lambda_max_gram(p.A, kappa, iters)
    else:
        lmax = 2.0 * lambda_max_gram(p.A, kappa, iters)   # Hess <= 2 A^T A
    return max(0.0, 0.5 * gamma * lmax * (1.0 + margin) - 1.0)
