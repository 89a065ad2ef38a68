"""Seeded generators for the synthetic workloads (problem data only).

Workloads follow the kinds of instance the paper experiments with (Section 4):

* ``nesterov_lasso``: a LASSO instance with a planted optimum, in the style of the
  Nesterov generator used for the paper's second LASSO test set (Section 4.2).  The
  paper only cites the generator, so the recipe below is this project's reading of it:

    1. y* ~ N(0, 1)^m (the dual point; at the optimum the residual is r* = -y*).
    2. B with entries iid U[-1, 1]; support S of size k drawn uniformly.
    3. s_j = b_j^T y*.  For j in S:  a_j = b_j * lam / |s_j| and
       x*_j = sign(s_j) * u_j with u_j ~ U(0, 1].
       For j not in S with |s_j| > lam:  a_j = b_j * lam * xi_j / |s_j| with
       xi_j ~ U(0, 1) (open), so that |a_j^T y*| < lam strictly.
       Other columns are kept as drawn (|a_j^T y*| <= lam already).
    4. b = y* + A x*.

  Then a_j^T y* = lam * sign(x*_j) on S and |a_j^T y*| < lam off S, which are the
  LASSO optimality conditions at x* with residual A x* - b = -y*, so
  F* = 0.5 ||y*||^2 + lam ||x*||_1 is known in closed form.  When A is stored in a
  lower precision than FP64, b is recomputed in FP64 from the *stored* A and then
  rounded, which keeps x* optimal up to the storage rounding of A.

* ``random_lasso``: unstructured dense instances (uniform or Gaussian entries), with
  optional zero columns, used for parity cases of arbitrary (ragged) shape.

* ``ncquad_problem``: the nonconvex quadratic of the form used in Section 4.3:
  A iid N(0, 1/m), x0 5% sparse with N(0, 1) entries, b = A x0 + 0.01 N(0, 1),
  box |x_i| <= 1.  The constant c of f = ||Ax - b||^2 - c||x||^2 and the weight lam
  are problem parameters chosen as documented on the function.

* ``liu_wright_lasso``: the Gaussian LASSO set of Section 4.2 (A iid N(0, 1), s-sparse
  xbar, b = A xbar + N(0, sigma^2) noise, lam = 20 sqrt(m log n) sigma).

* ``dc_problem``: the sparse-regression instance of Section 4.3's nonconvex experiment
  (F = ||Ax - b||^2 + lam H(x) with the log or exp regulariser): A with iid N(0, 1)
  entries and unit-norm columns, xbar 5% nonzero with N(0, 1) values, b = A xbar + e,
  e ~ N(0, 0.1^2).  lam is not given in the paper; it is a fixed fraction of the
  smallest weight for which x = 0 is stationary.
"""

from __future__ import annotations

import math

import numpy as np


def pad_lda(m: int, elt_bytes: int) -> int:
    """Smallest leading dimension >= m whose column stride is a multiple of 16 bytes."""
    per = max(1, 16 // elt_bytes)
    return ((m + per - 1) // per) * per


def _open_unit(rng: np.random.Generator, size) -> np.ndarray:
    """Uniform draws strictly inside (0, 1)."""
    u = rng.integers(0, 2 ** 52, size=size, dtype=np.int64).astype(np.float64)
    return (u + 0.5) / float(2 ** 52)


def nesterov_lasso(m: int, n: int, k: int, lam: float = 1.0, seed: int = 0,
                   store_dtype=np.float64, lda: int | None = None) -> dict:
    """Planted-optimum LASSO instance (numpy, FP64 construction).

    Returns a dict with
      At      (n, lda) array of ``store_dtype``; row j is column a_j (zero padded)
      b       (m,) array of ``store_dtype``
      x_star  (n,) FP64 planted minimiser
      y_star  (m,) FP64 dual point (residual at x_star is -y_star)
      f_star  FP64 closed-form optimal value 0.5||y*||^2 + lam ||x*||_1
      lam, m, n, lda, support
    """
    if not (0 <= k <= n):
        raise ValueError("support size out of range")
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(m)
    Bt = rng.uniform(-1.0, 1.0, size=(n, m))
    support = np.sort(rng.choice(n, size=k, replace=False)) if k > 0 else np.zeros(0, np.int64)
    mag = 1.0 - rng.uniform(0.0, 1.0, size=k)          # U(0, 1]
    xi = _open_unit(rng, n)                              # U(0, 1) open

    s = Bt @ y
    on = np.zeros(n, dtype=bool)
    on[support] = True
    if np.any(np.abs(s[on]) == 0.0):
        raise RuntimeError("degenerate draw: a support column is orthogonal to y*")
    scale = np.ones(n)
    scale[on] = lam / np.abs(s[on])
    big = (~on) & (np.abs(s) > lam)
    scale[big] = lam * xi[big] / np.abs(s[big])
    At64 = Bt * scale[:, None]

    x_star = np.zeros(n)
    x_star[support] = mag * np.sign(s[support])

    elt = np.dtype(store_dtype).itemsize
    if lda is None:
        lda = pad_lda(m, elt)
    At = np.zeros((n, lda), dtype=store_dtype)
    At[:, :m] = At64.astype(store_dtype)
    # b from the stored matrix, accumulated in FP64, then rounded to the storage type.
    stored = At[:, :m].astype(np.float64)
    b64 = y + stored[support].T @ x_star[support] if k > 0 else y.copy()
    b = b64.astype(store_dtype)
    f_star = 0.5 * float(y @ y) + lam * float(np.abs(x_star).sum())
    return dict(At=At, b=b, x_star=x_star, y_star=y, f_star=f_star, lam=float(lam),
                m=m, n=n, lda=lda, support=support, col_scale=scale)


def validation_rows(gen: dict, m_val: int, seed: int = 1, noise: float = 0.01) -> dict:
    """Validation split "from the same generator": m_val new rows with entries iid U[-1, 1]
    times the training column scalings, and b_val = A_val x* + noise * N(0, 1).
    Returns At_val (n, lda_val) in the training storage type and b_val."""
    rng = np.random.default_rng(seed)
    n = gen["n"]
    B = rng.uniform(-1.0, 1.0, size=(n, m_val)) * gen["col_scale"][:, None]
    dt = gen["At"].dtype
    lda = pad_lda(m_val, np.dtype(dt).itemsize)
    At_val = np.zeros((n, lda), dtype=dt)
    At_val[:, :m_val] = B.astype(dt)
    b_val = At_val[:, :m_val].astype(np.float64).T @ gen["x_star"] + noise * rng.standard_normal(m_val)
    return dict(At=At_val, b=b_val.astype(dt), m=m_val, n=n, lda=lda)


def nesterov_lasso_torch(m: int, n: int, k: int, lam: float = 1.0, seed: int = 0,
                         device="cuda", dtype=None, chunk: int = 4096, n_generate: int | None = None) -> dict:
    """Same recipe as :func:`nesterov_lasso`, generated with torch on ``device``.

    Used for instances too large to build on the host (e.g. 20000 x 100000).  The
    random stream differs from the numpy one, so instances are distinct but of the
    same distribution.  Construction is in FP64 column chunk by column chunk; the
    returned ``At`` is stored in ``dtype`` (default float32) with zero padding.
    Returns torch tensors on ``device`` (x_star, y_star in FP64).

    ``n_generate`` < n builds only the first n_generate columns (a bounded sample of the
    same draw): the support is restricted to those columns and b = y* + A x* uses them
    only, so the sample is itself a planted instance with n_generate variables.
    """
    import torch

    ncols = n if n_generate is None else min(n, int(n_generate))
    if dtype is None:
        dtype = torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    # the draws below always cover the full instance, so a sample is a prefix of it
    y = torch.randn(m, generator=g, device=device, dtype=f64)
    perm = torch.randperm(n, generator=g, device=device)
    support_full = torch.sort(perm[:k]).values
    mag_full = 1.0 - torch.rand(k, generator=g, device=device, dtype=f64)
    u = torch.randint(0, 2 ** 52, (n,), generator=g, device=device, dtype=torch.int64)
    xi = (u.to(f64) + 0.5) / float(2 ** 52)
    keep = support_full < ncols
    support = support_full[keep]
    mag = mag_full[keep]
    on = torch.zeros(ncols, dtype=torch.bool, device=device)
    on[support] = True

    elt = torch.tensor([], dtype=dtype).element_size()
    lda = pad_lda(m, elt)
    At = torch.zeros((ncols, lda), dtype=dtype, device=device)
    s_all = torch.empty(ncols, dtype=f64, device=device)
    col_scale = torch.empty(ncols, dtype=f64, device=device)
    for j0 in range(0, ncols, chunk):
        j1 = min(ncols, j0 + chunk)
        Bt = torch.rand((min(n, j0 + chunk) - j0, m), generator=g, device=device, dtype=f64)[: j1 - j0]
        Bt = Bt * 2.0 - 1.0
        s = Bt @ y
        s_all[j0:j1] = s
        o = on[j0:j1]
        sa = s.abs()
        scale = torch.ones(j1 - j0, dtype=f64, device=device)
        scale = torch.where(o, lam / sa, scale)
        big = (~o) & (sa > lam)
        scale = torch.where(big, lam * xi[j0:j1] / sa, scale)
        col_scale[j0:j1] = scale
        At[j0:j1, :m] = (Bt * scale[:, None]).to(dtype)
        del Bt
    ks = int(support.numel())
    if ks > 0 and bool((s_all[support] == 0).any()):
        raise RuntimeError("degenerate draw: a support column is orthogonal to y*")
    x_star = torch.zeros(ncols, dtype=f64, device=device)
    if ks:
        x_star[support] = mag * torch.sign(s_all[support])
    stored = At[support, :m].to(f64)
    b64 = y + stored.T @ x_star[support] if ks > 0 else y.clone()
    b = b64.to(dtype)
    f_star = 0.5 * float(y @ y) + lam * float(x_star.abs().sum())
    return dict(At=At, b=b, x_star=x_star, y_star=y, f_star=f_star, lam=float(lam),
                m=m, n=ncols, lda=lda, support=support, col_scale=col_scale)


def validation_rows_torch(gen: dict, m_val: int, seed: int = 1, noise: float = 0.01) -> dict:
    """:func:`validation_rows` for a torch instance (generated on its device)."""
    import torch

    dev = gen["At"].device
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    n = gen["n"]
    lda = pad_lda(m_val, gen["At"].element_size())
    At_val = torch.zeros((n, lda), dtype=gen["At"].dtype, device=dev)
    chunk = 8192
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        B = torch.rand((j1 - j0, m_val), generator=g, device=dev, dtype=torch.float64) * 2.0 - 1.0
        At_val[j0:j1, :m_val] = (B * gen["col_scale"][j0:j1, None]).to(gen["At"].dtype)
    sup = gen["support"]
    b_val = At_val[sup, :m_val].double().T @ gen["x_star"][sup] + noise * torch.randn(
        m_val, generator=g, device=dev, dtype=torch.float64)
    return dict(At=At_val, b=b_val.to(gen["At"].dtype), m=m_val, n=n, lda=lda)


def random_lasso(m: int, n: int, seed: int = 0, dist: str = "uniform", lam: float = 0.1,
                 store_dtype=np.float64, zero_cols: int = 0, lda: int | None = None,
                 box: float | None = None) -> dict:
    """Dense instance with iid entries (``uniform`` U[-1,1] or ``gauss`` N(0, 1/m)).

    ``zero_cols`` columns (chosen at random) are set exactly to zero, to exercise the
    degenerate-curvature case.  ``box`` gives symmetric bounds [-box, box] if set.
    b is iid N(0, 1).
    """
    rng = np.random.default_rng(seed)
    if dist == "uniform":
        At64 = rng.uniform(-1.0, 1.0, size=(n, m))
    elif dist == "gauss":
        At64 = rng.standard_normal((n, m)) / math.sqrt(max(m, 1))
    else:
        raise ValueError(dist)
    if zero_cols:
        zc = rng.choice(n, size=zero_cols, replace=False)
        At64[zc] = 0.0
    b64 = rng.standard_normal(m)
    elt = np.dtype(store_dtype).itemsize
    if lda is None:
        lda = pad_lda(m, elt)
    At = np.zeros((n, lda), dtype=store_dtype)
    At[:, :m] = At64.astype(store_dtype)
    out = dict(At=At, b=b64.astype(store_dtype), lam=float(lam), m=m, n=n, lda=lda)
    if box is not None:
        out["lo"] = np.full(n, -box, dtype=store_dtype)
        out["hi"] = np.full(n, box, dtype=store_dtype)
    return out


def ncquad_problem_torch(m: int, n: int, seed: int = 0, frac: float = 0.05, noise: float = 0.01,
                         box: float = 1.0, lam_frac: float = 0.3, device="cuda") -> dict:
    """:func:`ncquad_problem` generated with torch on ``device`` in FP32 storage (for the
    10000 x 50000 instance).  Same recipe; a different random stream."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lda = pad_lda(m, 4)
    At = torch.zeros((n, lda), dtype=torch.float32, device=device)
    chunk = 8192
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        At[j0:j1, :m] = torch.randn((j1 - j0, m), generator=g, device=device, dtype=torch.float32) / math.sqrt(m)
    k = int(round(frac * n))
    idx = torch.randperm(n, generator=g, device=device)[:k]
    x0 = torch.zeros(n, dtype=torch.float64, device=device)
    x0[idx] = torch.randn(k, generator=g, device=device, dtype=torch.float64)
    e = noise * torch.randn(m, generator=g, device=device, dtype=torch.float64)
    b64 = At[idx, :m].double().T @ x0[idx] + e
    b = b64.to(torch.float32)
    atb = torch.empty(n, dtype=torch.float64, device=device)
    for j0 in range(0, n, chunk):
        atb[j0:j0 + chunk] = At[j0:j0 + chunk, :m].double() @ b.double()
    c = 0.5 * (1.0 - math.sqrt(n / m)) ** 2
    lam = lam_frac * 2.0 * float(atb.abs().max())
    return dict(At=At, b=b, x0=x0, c=float(c), lam=float(lam), m=m, n=n, lda=lda,
                lo=torch.full((n,), -box, dtype=torch.float32, device=device),
                hi=torch.full((n,), box, dtype=torch.float32, device=device))


def liu_wright_lasso(m: int, n: int, s: int, sigma: float = 0.01, seed: int = 0, store_dtype=np.float64) -> dict:
    """The Gaussian LASSO set of Section 4.2: A with iid N(0, 1) entries, xbar with s nonzeros
    (iid N(0, 1) values at uniformly drawn positions), b = A xbar + e with e iid N(0, sigma^2),
    lam = 20 sqrt(m log n) sigma.  The optimum is not known in closed form."""
    rng = np.random.default_rng(seed)
    A64 = rng.standard_normal((n, m))
    xbar = np.zeros(n)
    idx = rng.choice(n, size=s, replace=False)
    xbar[idx] = rng.standard_normal(s)
    e = sigma * rng.standard_normal(m)
    elt = np.dtype(store_dtype).itemsize
    lda = pad_lda(m, elt)
    At = np.zeros((n, lda), dtype=store_dtype)
    At[:, :m] = A64.astype(store_dtype)
    b64 = At[:, :m].astype(np.float64).T @ xbar + e
    lam = 20.0 * math.sqrt(m * math.log(n)) * sigma
    return dict(At=At, b=b64.astype(store_dtype), xbar=xbar, lam=float(lam), m=m, n=n, lda=lda)


def liu_wright_lasso_torch(m: int, n: int, s: int, sigma: float = 0.01, seed: int = 0, device="cuda") -> dict:
    """:func:`liu_wright_lasso` generated with torch on ``device`` in FP32 storage; same recipe,
    a different random stream."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lda = pad_lda(m, 4)
    At = torch.zeros((n, lda), dtype=torch.float32, device=device)
    chunk = 8192
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        At[j0:j1, :m] = torch.randn((j1 - j0, m), generator=g, device=device, dtype=torch.float32)
    idx = torch.randperm(n, generator=g, device=device)[:s]
    xbar = torch.zeros(n, dtype=torch.float64, device=device)
    xbar[idx] = torch.randn(s, generator=g, device=device, dtype=torch.float64)
    e = sigma * torch.randn(m, generator=g, device=device, dtype=torch.float64)
    b = (At[idx, :m].double().T @ xbar[idx] + e).to(torch.float32)
    lam = 20.0 * math.sqrt(m * math.log(n)) * sigma
    return dict(At=At, b=b, xbar=xbar, lam=float(lam), m=m, n=n, lda=lda)


def dc_problem(m: int, n: int, reg: str = "log", theta: float = 20.0, seed: int = 0, frac: float = 0.05,
               sigma: float = 0.1, lam_frac: float = 0.1, store_dtype=np.float64) -> dict:
    """Sparse regression with a nonconvex regulariser (the log or exp penalty).

    A: iid N(0, 1) entries, each column scaled to unit norm; xbar: iid N(0, 1) with a random
    (1 - frac) of its entries set to 0; b = A xbar + e, e iid N(0, sigma^2).  ``theta`` is the
    regulariser parameter; lam = lam_frac * lam0 with lam0 = 2 ||A^T b||_inf / eta the
    smallest weight for which x = 0 is stationary (eta = theta for exp, theta / log(1 +
    theta) for log).  Returned ``loss`` is "dc_log" or "dc_exp" and ``c`` is unused.
    """
    rng = np.random.default_rng(seed)
    A64 = rng.standard_normal((n, m))
    A64 /= np.linalg.norm(A64, axis=1, keepdims=True)
    k = int(round(frac * n))
    xbar = np.zeros(n)
    if k:
        idx = rng.choice(n, size=k, replace=False)
        xbar[idx] = rng.standard_normal(k)
    e = sigma * rng.standard_normal(m)
    elt = np.dtype(store_dtype).itemsize
    lda = pad_lda(m, elt)
    At = np.zeros((n, lda), dtype=store_dtype)
    At[:, :m] = A64.astype(store_dtype)
    stored = At[:, :m].astype(np.float64)
    b64 = stored.T @ xbar + e
    eta = theta if reg == "exp" else theta / math.log1p(theta)
    lam = lam_frac * 2.0 * float(np.abs(stored @ b64.astype(store_dtype).astype(np.float64)).max()) / eta
    return dict(At=At, b=b64.astype(store_dtype), xbar=xbar, theta=float(theta), lam=float(lam),
                loss="dc_" + reg, c=0.0, m=m, n=n, lda=lda)


def dc_problem_torch(m: int, n: int, reg: str = "log", theta: float = 20.0, seed: int = 0, frac: float = 0.05,
                     sigma: float = 0.1, lam_frac: float = 0.1, device="cuda") -> dict:
    """:func:`dc_problem` generated with torch on ``device`` in FP32 storage; same recipe, a
    different random stream."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lda = pad_lda(m, 4)
    At = torch.zeros((n, lda), dtype=torch.float32, device=device)
    chunk = 8192
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        B = torch.randn((j1 - j0, m), generator=g, device=device, dtype=torch.float64)
        At[j0:j1, :m] = (B / B.norm(dim=1, keepdim=True)).to(torch.float32)
    k = int(round(frac * n))
    idx = torch.randperm(n, generator=g, device=device)[:k]
    xbar = torch.zeros(n, dtype=torch.float64, device=device)
    xbar[idx] = torch.randn(k, generator=g, device=device, dtype=torch.float64)
    e = sigma * torch.randn(m, generator=g, device=device, dtype=torch.float64)
    b = (At[idx, :m].double().T @ xbar[idx] + e).to(torch.float32)
    atb = torch.empty(n, dtype=torch.float64, device=device)
    for j0 in range(0, n, chunk):
        atb[j0:j0 + chunk] = At[j0:j0 + chunk, :m].double() @ b.double()
    eta = theta if reg == "exp" else theta / math.log1p(theta)
    lam = lam_frac * 2.0 * float(atb.abs().max()) / eta
    return dict(At=At, b=b, xbar=xbar, theta=float(theta), lam=float(lam), loss="dc_" + reg, c=0.0,
                m=m, n=n, lda=lda)


def ncquad_problem(m: int, n: int, seed: int = 0, frac: float = 0.05, noise: float = 0.01,
                   box: float = 1.0, lam_frac: float = 0.3, store_dtype=np.float64) -> dict:
    """Nonconvex quadratic instance  f = ||Ax - b||^2 - c||x||^2,  G = lam||x||_1, |x| <= box.

    A iid N(0, 1/m); x0 has round(frac * n) nonzeros drawn N(0, 1); b = A x0 + noise N(0,1).
    c = 0.5 * (1 - sqrt(n/m))^2 (half the lower edge of the Marchenko-Pastur law of the
    nonzero spectrum of A^T A), which makes f nonconvex on the null space of A while
    every coordinate curvature 2||a_j||^2 - 2c stays positive for the usual draw.
    lam = lam_frac * 2 ||A^T b||_inf (lam_frac times the smallest weight for which
    x = 0 is stationary).  The default 0.3 puts lam above 2c on the usual shapes, so the
    penalty lam|x| - c x^2 still increases on the box (a nonconvex, MCP-like penalty); with
    lam < 2c the concave term drives most coordinates to the box over thousands of sweeps.
    """
    rng = np.random.default_rng(seed)
    At64 = rng.standard_normal((n, m)) / math.sqrt(m)
    k = int(round(frac * n))
    x0 = np.zeros(n)
    if k:
        idx = rng.choice(n, size=k, replace=False)
        x0[idx] = rng.standard_normal(k)
    e = noise * rng.standard_normal(m)
    elt = np.dtype(store_dtype).itemsize
    lda = pad_lda(m, elt)
    At = np.zeros((n, lda), dtype=store_dtype)
    At[:, :m] = At64.astype(store_dtype)
    stored = At[:, :m].astype(np.float64)
    b64 = stored.T @ x0 + e
    c = 0.5 * (1.0 - math.sqrt(n / m)) ** 2
    lam = lam_frac * 2.0 * float(np.abs(stored @ b64).max())
    return dict(At=At, b=b64.astype(store_dtype), x0=x0, c=float(c), lam=float(lam),
                lo=np.full(n, -box, dtype=store_dtype), hi=np.full(n, box, dtype=store_dtype),
                m=m, n=n, lda=lda)
