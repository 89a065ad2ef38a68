"""Pins for the multi-core CPU oracle (oracle/cores.c): the partitioned lock-free form of
Algorithm 1 for LASSO on host threads, used for the core-count study of Section 4.2.

* One thread is the cyclic block Gauss-Seidel method: same iterates as the numpy oracle, in
  both forms (threads sharing the residual, or sharing x with A^T A precomputed).
* Any number of threads converges to the exact LASSO minimiser found by enumerating sign
  patterns (tiny n), and to the planted closed-form optimum of the Nesterov generator.
* The stopping rule is the relative error of F against F* (Section 4.2).
"""

import math
import shutil

import numpy as np
import pytest

import oracle as O
from inputs import nesterov_lasso

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed to build the C oracle")


def _cores():
    from oracle import cores
    return cores


def _fp32_problem(d):
    """The generator's data with A and b as stored in FP32, as numpy FP64 oracle data."""
    d = dict(d)
    d["At"] = np.asarray(d["At"], dtype=np.float32)
    return d, O.Problem.from_data(d)


def _form(d, form):
    if form == "residual":
        return {}
    Q, q = _cores().gram(d["At"], d["b"], d["m"])
    return {"Q": Q, "q": q}


@pytest.mark.parametrize("form", ["residual", "gram"])
@pytest.mark.parametrize("w", [1, 4, 7])
def test_one_thread_equals_gauss_seidel(w, form):
    d, p = _fp32_problem(nesterov_lasso(200, 1000, 50, lam=1.0, seed=1, store_dtype=np.float32))
    x, st = _cores().partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], gamma=0.9, tau=0.5, w=w, threads=1,
                                       max_sweeps=3, **_form(d, form))
    dw = O.surrogate_weights(p, tau=0.5)
    xr = np.zeros(p.n)
    rr = O.residual(p, xr)
    for _ in range(3):
        xr, rr = O.gauss_seidel_sweep(p, xr, rr, dw, 0.9, w=w)
    assert st["sweeps"] == 3 and st["block_updates"] == 3 * math.ceil(p.n / w)
    assert np.abs(x - xr).max() <= (1e-12 if form == "residual" else 1e-10) * np.abs(xr).max()
    assert abs(st["F"] - O.objective(p, xr)) <= 1e-12 * abs(st["F"])
    assert abs(st["F_running"] - st["F"]) <= 1e-12 * abs(st["F"])


@pytest.mark.parametrize("form", ["residual", "gram"])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_reaches_brute_force_minimiser(threads, form):
    rng = np.random.default_rng(5)
    m, n = 30, 8
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m)
    lam = 0.3 * float(np.abs(A.astype(np.float64).T @ b).max())
    found = O.brute_force_lasso(A.astype(np.float64), b, lam)
    assert len(found) == 1
    xs = found[0]
    assert 0 < np.count_nonzero(xs) < n  # both zero and nonzero coordinates are exercised
    At = np.ascontiguousarray(A.T)
    x, st = _cores().partitioned_lasso(At, b, m, lam, gamma=0.9, w=1, threads=threads, max_sweeps=3000,
                                       **_form({"At": At, "b": b, "m": m}, form))
    assert st["block_updates"] == st["sweeps"] * n  # each block owned by exactly one thread (D4)
    assert np.abs(x - xs).max() <= 1e-9 * max(1.0, np.abs(xs).max())


@pytest.mark.parametrize("form", ["residual", "gram"])
def test_partitioned_threads_reach_planted_optimum(form):
    """Nesterov instance stored in FP32 (b recomputed from the stored A): the closed-form
    optimum holds to about FP32 rounding, so the stop at 1e-6 relative error is reached and
    every thread count lands on the same minimiser."""
    d, p = _fp32_problem(nesterov_lasso(300, 1200, 40, lam=1.0, seed=2, store_dtype=np.float32))
    f_star = d["f_star"]
    fm = _form(d, form)
    xs = []
    for threads in (1, 4):
        x, st = _cores().partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], gamma=0.9, w=1, threads=threads,
                                           max_sweeps=2000, f_star=f_star, tol=1e-6, **fm)
        assert st["sweeps"] < 2000 and st["block_updates"] == st["sweeps"] * p.n
        assert (st["F_running"] - f_star) / f_star < 1e-6
        assert abs(st["F"] - O.objective(p, x)) <= 1e-12 * st["F"]
        assert (st["F"] - f_star) / f_star < 1.1e-6
        x, _ = _cores().partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], gamma=0.9, w=1, threads=threads,
                                          max_sweeps=3000, x0=x, **fm)
        xs.append(x)
    assert np.abs(xs[0] - xs[1]).max() <= 1e-6
    assert np.abs(xs[0] - d["x_star"]).max() <= 1e-3  # FP32 storage moves the minimiser slightly


def test_stop_is_the_first_sweep_below_tol():
    d, p = _fp32_problem(nesterov_lasso(200, 800, 30, lam=1.0, seed=3, store_dtype=np.float32))
    f_star = d["f_star"]
    c = _cores()
    _, st = c.partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], threads=1, max_sweeps=1000, f_star=f_star,
                                tol=1e-4)
    k = st["sweeps"]
    assert k > 1 and (st["F_running"] - f_star) / f_star < 1e-4
    _, st1 = c.partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], threads=1, max_sweeps=k - 1, f_star=f_star,
                                 tol=1e-4)
    assert st1["sweeps"] == k - 1 and (st1["F_running"] - f_star) / f_star >= 1e-4
    _, st2 = c.partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], threads=1, max_sweeps=1000, f_star=f_star,
                                 tol=1e-7)
    assert st2["sweeps"] > k


@pytest.mark.parametrize("kw", [{"threads": 0}, {"w": 0}, {"max_sweeps": -1}, {"Q": np.eye(40)},
                                {"Q": np.eye(39), "q": np.zeros(39)}])
def test_bad_arguments_raise(kw):
    d = nesterov_lasso(20, 40, 4, seed=0, store_dtype=np.float32)
    args = dict(threads=1, w=1, max_sweeps=1)
    args.update(kw)
    with pytest.raises(ValueError):
        _cores().partitioned_lasso(d["At"], d["b"], d["m"], d["lam"], **args)
