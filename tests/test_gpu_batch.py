"""Batched form: many problems in one sweep launch per round (CUDA-graph rounds)."""

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
    bs = BatchSolver([_cuda(d) for d in ds], block_w=8, num_ctas=1, refresh_every=2, max_sweeps=2)
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
    bs = BatchSolver([_cuda(d) for d in ds], block_w=16, num_ctas=16, refresh_every=5, max_sweeps=4000)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for d in ds]
    per, tot = bs.solve(xs, f_star=f_ref)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for i in (0, 5):
        p = O.Problem.from_data(ds[i])
        F = O.objective(p, xs[i].cpu().numpy().astype(np.float64))
        assert (F - f_ref[i]) / f_ref[i] <= 1.5e-6
        assert abs(F - per[i]["F"]) <= 1e-9 * F
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
                     shared_a=True)
    xs = [torch.zeros(d["n"], dtype=torch.float32, device="cuda") for _ in lams]
    per, tot = bs.solve(xs)
    assert tot["block_w"] in (16, 32, 64)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for k, lam in enumerate(lams):
        p = O.Problem.from_data(d)
        p.lam = lam
        xk = xs[k].cpu().numpy().astype(np.float64)
        merit = O.stationarity(O.xhat_merit(p, xk, O.surrogate_weights(p)), xk)
        assert merit <= 1e-4, (lam, merit)
    # the lambda = 1 lane reaches the planted optimum
    p = O.Problem.from_data(d)
    f1 = O.objective(p, d["x_star"])
    assert (O.objective(p, xs[3].cpu().numpy().astype(np.float64)) - f1) / f1 <= 1e-5
    bs.close()
