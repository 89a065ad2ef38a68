"""Batched forms, through the C ABI, against the FP64 oracle.

* Gauss-Seidel form: one persistent launch, one CTA per problem at a time; its iterates are
  exact cyclic coordinate Gauss-Seidel sweeps, and every problem stops at the gap and
  stationarity tolerances (checked by the oracle at the returned x).
* Async rounds: one sweep launch per round over all problems' blocks (CUDA-graph rounds);
  a problem that leaves the rounds is held to the same stationarity by an exact check.
"""

import numpy as np
import pytest

import oracle as O
from inputs import nesterov_lasso, random_lasso
from tests._gpu_helpers import rel_inf

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1701_04900_gb300.build import build_library
    build_library()


def _cuda(d):
    import torch
    return dict(At=torch.from_numpy(np.ascontiguousarray(d["At"])).cuda(), b=torch.from_numpy(d["b"]).cuda(),
                lam=d["lam"], m=d["m"])


def test_batch_single_cta_is_gauss_seidel_per_problem():
    """One CTA walks the global block list in order, so each (independent) problem sees a
    cyclic block Gauss-Seidel sweep of its own blocks."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    shapes = [(301, 120), (1003, 77), (64, 200)]
    ds = [random_lasso(m, n, seed=50 + i, lam=0.2, store_dtype=np.float32) for i, (m, n) in enumerate(shapes)]
    bs = BatchSolver([_cuda(d) for d in ds], block_w=8, num_ctas=1, refresh_every=2, max_sweeps=2, form="async")
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs)
    assert tot["sweeps"] == 2
    for d, x in zip(ds, xs):
        p = O.Problem.from_data(d)
        dw = O.surrogate_weights(p)
        xr, rr = np.zeros(p.n), O.residual(p, np.zeros(p.n))
        for _ in range(2):
            xr, rr = O.gauss_seidel_sweep(p, xr, rr, dw, 0.9, w=8)
        assert rel_inf(x.cpu().numpy(), xr) < TOL32
    bs.close()


def test_batch_uneven_instances_reach_their_optima():
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    rng = np.random.default_rng(7)
    ds = []
    for i in range(8):
        m = int(rng.integers(300, 1500))
        n = int(rng.integers(1000, 5000))
        ds.append(nesterov_lasso(m, n, max(1, n // 50), lam=1.0, seed=60 + i, store_dtype=np.float32))
    f_ref = [O.objective(O.Problem.from_data(d), d["x_star"]) for d in ds]
    bs = BatchSolver([_cuda(d) for d in ds], block_w=16, num_ctas=16, refresh_every=5, max_sweeps=4000,
                     form="async")
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs, f_star=f_ref)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for i in range(len(ds)):
        p = O.Problem.from_data(ds[i])
        xi = xs[i].cpu().numpy().astype(np.float64)
        F = O.objective(p, xi)
        assert (F - f_ref[i]) / f_ref[i] <= 1.5e-6
        assert abs(F - per[i]["F"]) <= 1e-9 * F
        assert O.stationarity(O.xhat_merit(p, xi, O.surrogate_weights(p)), xi) <= 1.5e-6
    assert all(s["rel_gap"] <= 1.5e-6 for s in per)
    bs.close()


def test_batch_shared_matrix_lambda_path_with_autotuned_width():
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    d = nesterov_lasso(1000, 4000, 40, lam=1.0, seed=70, store_dtype=np.float32)
    base = _cuda(d)
    lams = [4.0, 2.0, 1.5, 1.0]
    probs = [dict(base, lam=l) for l in lams]
    bs = BatchSolver(probs, block_w=0, num_ctas=16, refresh_every=5, max_sweeps=4000, switch_tol=1e-10,
                     shared_a=True, form="async")
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for _ in lams]
    per, tot = bs.solve(xs)
    assert tot["block_w"] in (16, 32, 64)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for k, lam in enumerate(lams):
        p = O.Problem.from_data(d)
        p.lam = lam
        xk = xs[k].cpu().numpy().astype(np.float64)
        merit = O.stationarity(O.xhat_merit(p, xk, O.surrogate_weights(p)), xk)
        assert merit <= 1.5e-6, (lam, merit)
    # the lambda = 1 lane reaches the planted optimum
    p = O.Problem.from_data(d)
    f1 = O.objective(p, d["x_star"])
    assert (O.objective(p, xs[3].cpu().numpy().astype(np.float64)) - f1) / f1 <= 1e-5
    bs.close()


# ----------------------------------------------------------------------------- Gauss-Seidel form

def _gs_oracle_sweeps(d, sweeps, gamma=0.9, w=1, x0=None):
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p)
    x = np.zeros(p.n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = O.residual(p, x)
    for _ in range(sweeps):
        x, r = O.gauss_seidel_sweep(p, x, r, dw, gamma, w=w)
    return x


@pytest.mark.parametrize("w", [1, 4, 8])
def test_batch_gs_form_iterates_are_block_gauss_seidel(w):
    """No stopping possible (tol_stat = 0, 2 sweeps in all): each problem's x equals two
    cyclic block Gauss-Seidel sweeps (blocks of w columns, w = 1: scalar blocks) of the oracle.
    Shapes cover a partial last unit (m = 5, 301), a single column (n = 1: the producer stays at
    most one column ahead), n below the ring depth and below w, n not a multiple of w, and the
    longest columns of the form's 15-warp shape."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    from paper_1701_04900_gb300 import native
    shapes = [(301, 121), (1003, 77), (64, 200), (4000, 50), (5, 3), (777, 1), (300, 22), (8192, 41)]
    ds = [random_lasso(m, n, seed=80 + i, lam=0.2, store_dtype=np.float32) for i, (m, n) in enumerate(shapes)]
    bs = BatchSolver([_cuda(d) for d in ds], form="gs", block_w=w, max_sweeps=2, check_every=2, tol_stat=0.0)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs)
    assert tot["batch_form"] == native.BATCH_FORM_GS and tot["block_w"] == w
    assert tot["ctas_per_sm"] >= 1
    for d, x, st in zip(ds, xs, per):
        # a problem uses fewer columns per block if a ring slot holds fewer of its columns
        assert 1 <= st["block_w"] <= w
        assert st["sweeps"] == 2 and st["status"] == native.ENOTCONV
        assert rel_inf(x.cpu().numpy(), _gs_oracle_sweeps(d, 2, w=st["block_w"])) < TOL32
    assert any(st["block_w"] == w for st in per)
    bs.close()


@pytest.mark.parametrize("w", [2, 4, 8])
def test_batch_gs_form_warm_start_with_a_refresh_every_sweep(w):
    """From a nonzero x0 (every third coordinate nonzero) with a check after every sweep, the
    residual the kernel starts each sweep from is rebuilt from x over the blocks that hold a
    nonzero: x after 3 sweeps equals 3 oracle block Gauss-Seidel sweeps from x0.  Columns of
    m = 1200 and 1700 (3 and 2 to a 16 KB ring slot) and 2400 and 3000 (3 and 2 to a 32 KB
    slot) give blocks narrower than w whichever slot the autotuner takes, so the rebuild's
    blocks do not line up with its groups of 32 columns."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    from paper_1701_04900_gb300 import native
    shapes = [(1200, 100), (1700, 70), (2400, 50), (3000, 40), (301, 121), (4000, 45), (64, 33)]
    ds = [random_lasso(m, n, seed=120 + i, lam=0.2, store_dtype=np.float32) for i, (m, n) in enumerate(shapes)]
    x0s = []
    for i, d in enumerate(ds):
        v = np.random.default_rng(300 + i).uniform(-0.5, 0.5, d["n"]).astype(np.float32)
        v[np.arange(d["n"]) % 3 != 0] = 0.0
        x0s.append(v)
    bs = BatchSolver([_cuda(d) for d in ds], form="gs", block_w=w, max_sweeps=3, check_every=1, tol_stat=0.0)
    xs = [torch.from_numpy(v.copy()).cuda() for v in x0s]
    per, _ = bs.solve(xs)
    for d, v, x, st in zip(ds, x0s, xs, per):
        assert st["sweeps"] == 3 and st["status"] == native.ENOTCONV
        ref = _gs_oracle_sweeps(d, 3, w=st["block_w"], x0=v)
        assert rel_inf(x.cpu().numpy(), ref) < TOL32, (d["m"], d["n"], st["block_w"])
    widths = {st["block_w"] for st in per[:4]}
    # a width that does not divide 32 (3 or 6)
    assert any(32 % wb for wb in widths) if w > 2 else widths <= {1, 2}
    bs.close()


def _fp32_floor(p):
    """The merit of the oracle's FP64 optimum rounded to FP32: what an FP32 iterate can reach."""
    x, _, _ = O.solve_gs(p, gamma=0.9, w=32, max_sweeps=400, tol=1e-15)
    x32 = x.astype(np.float32).astype(np.float64)
    return O.stationarity(O.xhat_merit(p, x32, O.surrogate_weights(p)), x32)


def test_batch_gs_form_uneven_instances_reach_gap_and_stationarity():
    """24 planted Nesterov instances of uneven sizes in one launch: every problem stops with
    the relative gap <= 1e-6 and ||xhat(x) - x||_inf / max(1, ||x||_inf) <= 1e-6, confirmed by
    the oracle at the returned x (1.5e-6 allows for the FP32 iterate), and the library's
    exact check agrees with the in-kernel one.  A problem whose FP32 iterate cannot reach
    1e-6 (the generator's column norms span up to 8 decades) stops at its floor (ENOTCONV):
    then the oracle's FP64 optimum rounded to FP32 is itself above 7.5e-7 and the returned x
    is within 2x of it."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    rng = np.random.default_rng(9)
    ds = []
    for i in range(24):
        m = int(rng.integers(300, 3000))
        n = int(rng.integers(1000, 6000))
        ds.append(nesterov_lasso(m, n, max(1, n // 50), lam=1.0, seed=90 + i, store_dtype=np.float32))
    f_ref = [O.objective(O.Problem.from_data(d), d["x_star"]) for d in ds]
    bs = BatchSolver([_cuda(d) for d in ds], form="gs", max_sweeps=3000, check_every=10)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs, f_star=f_ref)
    assert all(s["status"] in (0, 1) for s in per), [s["status"] for s in per]
    assert sum(s["status"] == 0 for s in per) >= 18
    exact = bs.check(xs, f_star=f_ref)
    for i, d in enumerate(ds):
        p = O.Problem.from_data(d)
        xi = xs[i].cpu().numpy().astype(np.float64)
        F = O.objective(p, xi)
        assert (F - f_ref[i]) / f_ref[i] <= 1.5e-6
        assert abs(F - per[i]["F"]) <= 1e-9 * F
        merit = O.stationarity(O.xhat_merit(p, xi, O.surrogate_weights(p)), xi)
        assert abs(exact[i]["stat_xhat"] - merit) <= 2e-7 * max(1.0, merit / 1e-6)
        if per[i]["status"] == 0:
            assert merit <= 1.5e-6, (i, merit, per[i]["stat_xhat"])
        else:
            floor = _fp32_floor(p)
            assert floor > 7.5e-7 and merit <= 2.0 * floor, (i, merit, floor)
    bs.close()


def test_batch_gs_form_hands_slow_problems_to_further_launches():
    """Problems still short of their tolerances after 300 sweeps leave the first launch and
    continue from their iterates in further launches (their own tuned shape): they report
    the sweeps of every launch, the handoff count, and, when they stop with OK, the gap and
    the stationarity the oracle confirms; the quick problems finish in the first launch."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    ds = [nesterov_lasso(1200, 3000, 60, lam=1.0, seed=140 + i, store_dtype=np.float32) for i in range(3)]
    ds += [nesterov_lasso(300, 7000, 150, lam=1.0, seed=150 + i, store_dtype=np.float32) for i in range(3)]
    f_ref = [O.objective(O.Problem.from_data(d), d["x_star"]) for d in ds]
    bs = BatchSolver([_cuda(d) for d in ds], form="gs", max_sweeps=3000, check_every=10)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs, f_star=f_ref)
    handed = [i for i, st in enumerate(per) if st["handed_over"] > 0]
    assert tot["handed_over"] == len(handed) >= 1, [st["sweeps"] for st in per]
    for i, st in enumerate(per):
        assert st["status"] in (0, 1)
        if i in handed:
            assert st["sweeps"] > 300
        else:
            assert st["sweeps"] <= 310
        if st["status"] == 1:
            continue
        p = O.Problem.from_data(ds[i])
        xi = xs[i].cpu().numpy().astype(np.float64)
        F = O.objective(p, xi)
        assert (F - f_ref[i]) / f_ref[i] <= 1.5e-6
        assert abs(F - st["F"]) <= 1e-9 * F
        assert O.stationarity(O.xhat_merit(p, xi, O.surrogate_weights(p)), xi) <= 1.5e-6, i
    assert any(per[i]["status"] == 0 for i in handed)
    bs.close()


def test_batch_gs_form_finishes_the_last_few_problems_with_the_async_solver():
    """With a budget of 1500 sweeps, problems still short of their tolerances after the first
    launch's 300 sweeps would run in one further launch to the budget; there are at most four of
    them, so each is finished by the single-problem async solver instead.  They report the async
    form, the sweeps of both parts, and, when they stop with OK, the gap and stationarity the
    oracle confirms at the returned x; the quick problems stay in the Gauss-Seidel form."""
    import torch
    from paper_1701_04900_gb300 import native
    from paper_1701_04900_gb300.batch import BatchSolver
    ds = [nesterov_lasso(1200, 3000, 60, lam=1.0, seed=140 + i, store_dtype=np.float32) for i in range(3)]
    ds += [nesterov_lasso(300, 7000, 150, lam=1.0, seed=150 + i, store_dtype=np.float32) for i in range(3)]
    f_ref = [O.objective(O.Problem.from_data(d), d["x_star"]) for d in ds]
    bs = BatchSolver([_cuda(d) for d in ds], form="gs", max_sweeps=1500, check_every=10)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs, f_star=f_ref)
    handed = [i for i, st in enumerate(per) if st["handed_over"] > 0]
    assert 1 <= len(handed) <= 4 and tot["handed_over"] == len(handed), [st["sweeps"] for st in per]
    for i, st in enumerate(per):
        assert st["status"] in (0, 1)
        if i in handed:
            assert st["batch_form"] == native.BATCH_FORM_ASYNC and 300 < st["sweeps"] <= 1500
        else:
            assert st["batch_form"] == native.BATCH_FORM_GS and st["sweeps"] <= 310
        if st["status"] == 1:
            continue
        p = O.Problem.from_data(ds[i])
        xi = xs[i].cpu().numpy().astype(np.float64)
        F = O.objective(p, xi)
        assert (F - f_ref[i]) / f_ref[i] <= 1.5e-6, i
        assert abs(F - st["F"]) <= 1e-9 * F
        assert O.stationarity(O.xhat_merit(p, xi, O.surrogate_weights(p)), xi) <= 1.5e-6, i
    assert any(per[i]["status"] == 0 for i in handed)
    bs.close()


def test_batch_shared_matrix_lambda_path_takes_the_multi_lane_form():
    """Problems that share A (a lambda path, shared_a) go to the multi-lane form by default:
    every lane exactly stationary to 1e-6 (oracle-confirmed to 1.5e-6), the iterates written
    back to each problem's x, and the planted lane at its optimum."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    from paper_1701_04900_gb300 import native
    d = nesterov_lasso(1000, 4000, 40, lam=1.0, seed=71, store_dtype=np.float32)
    base = _cuda(d)
    lams = [6.0, 3.0, 2.0, 1.4, 1.0]
    bs = BatchSolver([dict(base, lam=l) for l in lams], shared_a=True, max_sweeps=3000, tol_stat=1e-6)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for _ in lams]
    p1 = O.Problem.from_data(d)
    f1 = O.objective(p1, d["x_star"])
    per, tot = bs.solve(xs, f_star=[float("nan")] * 4 + [f1])
    assert tot["batch_form"] == native.BATCH_FORM_MULTI and tot["status"] == 0, tot
    for k, lam in enumerate(lams):
        assert per[k]["batch_form"] == native.BATCH_FORM_MULTI
        p = O.Problem.from_data(d)
        p.lam = lam
        xk = xs[k].cpu().numpy().astype(np.float64)
        merit = O.stationarity(O.xhat_merit(p, xk, O.surrogate_weights(p)), xk)
        assert per[k]["stat_xhat"] <= 1e-6 and merit <= 1.5e-6, (lam, merit)
    assert (O.objective(p1, xs[-1].cpu().numpy().astype(np.float64)) - f1) / f1 <= 1.5e-6
    bs.close()


def test_batch_gs_form_shared_matrix_lambda_path_and_cached_shape():
    """A lambda path on one matrix (f_star unknown: the problems stop on the merit alone);
    every lane is stationary to 1e-6 by the oracle, and the lambda = 1 lane reaches the
    planted optimum.  A second batch of the same shape reuses the tuned launch shape (no
    tuning sweeps)."""
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    d = nesterov_lasso(1000, 4000, 40, lam=1.0, seed=71, store_dtype=np.float32)
    base = _cuda(d)
    lams = [4.0, 2.0, 1.5, 1.0]
    probs = [dict(base, lam=l) for l in lams]
    bs = BatchSolver(probs, form="gs", shared_a=True, max_sweeps=3000, check_every=5)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for _ in lams]
    per, tot = bs.solve(xs)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for k, lam in enumerate(lams):
        p = O.Problem.from_data(d)
        p.lam = lam
        xk = xs[k].cpu().numpy().astype(np.float64)
        merit = O.stationarity(O.xhat_merit(p, xk, O.surrogate_weights(p)), xk)
        assert merit <= 1.5e-6, (lam, merit)
    p = O.Problem.from_data(d)
    f1 = O.objective(p, d["x_star"])
    assert (O.objective(p, xs[3].cpu().numpy().astype(np.float64)) - f1) / f1 <= 1.5e-6
    bs.close()
    # same shape: the cached launch shape, so the solve is the one launch (no tuning launches)
    bs2 = BatchSolver(probs, form="gs", shared_a=True, max_sweeps=3000, check_every=5)
    per2, tot2 = bs2.solve(xs)
    assert tot2["status"] == 0
    assert tot2["kernel_launches"] == 1
    assert tot2["ctas_per_sm"] == tot["ctas_per_sm"] and tot2["block_w"] == tot["block_w"]
    bs2.close()


def test_batch_gs_form_nonconvex_quadratic_with_box_is_stationary():
    import torch
    from inputs import ncquad_problem
    from paper_1701_04900_gb300.batch import BatchSolver
    ds = [ncquad_problem(800 + 200 * i, 2400 + 400 * i, seed=33 + i, store_dtype=np.float32) for i in range(3)]
    probs = []
    for d in ds:
        t = _cuda(d)
        t.update(lo=torch.from_numpy(d["lo"]).cuda(), hi=torch.from_numpy(d["hi"]).cuda(), loss="ncquad", c=d["c"])
        probs.append(t)
    bs = BatchSolver(probs, form="gs", max_sweeps=4000, check_every=10)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for d, x, st in zip(ds, xs, per):
        p = O.Problem.from_data(d, loss="ncquad")
        xg = x.cpu().numpy().astype(np.float64)
        assert np.all(xg >= -1.0) and np.all(xg <= 1.0)
        merit = O.stationarity(O.xhat_merit(p, xg, O.surrogate_weights(p)), xg)
        assert merit <= 1.5e-6
        assert abs(O.objective(p, xg) - st["F"]) <= 1e-9 * max(1.0, abs(st["F"]))
    bs.close()


def test_batch_gs_form_nan_is_reported():
    """A NaN in one problem's b: that problem ends with ENONFINITE, the others converge."""
    import torch
    from paper_1701_04900_gb300 import native
    from paper_1701_04900_gb300.batch import BatchSolver
    ds = [nesterov_lasso(300, 900, 18, lam=1.0, seed=110 + i, store_dtype=np.float32) for i in range(3)]
    ds[1]["b"] = ds[1]["b"].copy()
    ds[1]["b"][7] = np.nan
    bs = BatchSolver([_cuda(d) for d in ds], form="gs", max_sweeps=3000, check_every=10)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs)
    assert per[1]["status"] == native.ENONFINITE
    assert per[0]["status"] == 0 and per[2]["status"] == 0, (per[0], per[2])
    assert tot["status"] == native.ENONFINITE
    bs.close()
