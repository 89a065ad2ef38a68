"""Multi-lane form: k LASSO lanes sharing A, block updates of all lanes on the tensor cores."""

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


def _lanes(d, bs, lams):
    import torch
    At = torch.from_numpy(np.ascontiguousarray(d["At"])).cuda()
    B = torch.from_numpy(np.ascontiguousarray(np.stack(bs).astype(np.float32))).cuda()
    return At, B


@pytest.mark.parametrize("m,n,k", [(777, 300, 5), (1500, 200, 8), (300, 129, 1)])
def test_multi_single_cta_is_gauss_seidel_per_lane(m, n, k):
    """One CTA walks the blocks in order, so every lane sees cyclic Gauss-Seidel sweeps of its
    own problem (A, b_l, lam_l); the products are FP32-grade (TF32 hi/lo split)."""
    import torch
    from paper_1701_04900_gb300.batch import MultiLaneSolver
    d = random_lasso(m, n, seed=m + n, lam=0.1, dist="gauss", store_dtype=np.float32)
    rng = np.random.default_rng(k)
    bs = [d["b"].astype(np.float64) + 0.3 * l * rng.standard_normal(m) for l in range(k)]
    bs = [b.astype(np.float32) for b in bs]
    lams = [0.05 + 0.07 * l for l in range(k)]
    At, B = _lanes(d, bs, lams)
    ms = MultiLaneSolver(At, B, lams, m, num_ctas=1, max_sweeps=3, check_every=3, refresh_every=100,
                         tol_stat=0.0, tol_gap=0.0)
    X = torch.zeros((k, n), dtype=torch.float32, device="cuda")
    ms.solve(X)
    for l in range(k):
        p = O.Problem(A=d["At"][:, :m].astype(np.float64).T, b=bs[l].astype(np.float64), lam=lams[l])
        dw = O.surrogate_weights(p)
        x, r = np.zeros(n), O.residual(p, np.zeros(n))
        for _ in range(3):
            x, r = O.gauss_seidel_sweep(p, x, r, dw, 0.9, w=32)
        assert rel_inf(X[l].cpu().numpy(), x) < TOL32, l
    ms.close()


def test_multi_lambda_path_reaches_the_optimum():
    """A lambda path on a planted instance: every lane stops at stationarity <= 1e-6 as the
    library's exact check measures it (the tensor-core gradients only decide when to check),
    the FP64 oracle confirms it (1.5e-6 allows for the FP32 iterate; the library's figure
    agrees with the oracle's to 2e-8), and the lambda = 1 lane reaches the planted optimum."""
    import torch
    from paper_1701_04900_gb300.batch import MultiLaneSolver
    d = nesterov_lasso(1000, 4000, 40, lam=1.0, seed=70, store_dtype=np.float32)
    lams = [8.0, 4.0, 2.0, 1.5, 1.2, 1.0]
    At, B = _lanes(d, [d["b"]] * len(lams), lams)
    p1 = O.Problem.from_data(d)
    f1 = O.objective(p1, d["x_star"])
    fs = [None] * (len(lams) - 1) + [f1]
    ms = MultiLaneSolver(At, B, lams, d["m"], max_sweeps=3000, check_every=10, refresh_every=10, tol_stat=1e-6)
    X = torch.zeros((len(lams), d["n"]), dtype=torch.float32, device="cuda")
    per, tot = ms.solve(X, f_star=fs)
    assert tot["status"] == 0, (tot, [s["status"] for s in per])
    for l, lam in enumerate(lams):
        p = O.Problem.from_data(d)
        p.lam = lam
        x = X[l].cpu().numpy().astype(np.float64)
        merit = O.stationarity(O.xhat_merit(p, x, O.surrogate_weights(p)), x)
        assert merit <= 1.5e-6, (lam, merit)
        assert per[l]["stat_xhat"] <= 1e-6
        assert abs(per[l]["stat_xhat"] - merit) <= 2e-8, (lam, per[l]["stat_xhat"], merit)
        assert O.objective(p, x) == pytest.approx(per[l]["F"], rel=1e-9)
    assert (per[-1]["F"] - f1) / f1 <= 1e-6
    ms.close()


def test_multi_many_lanes_padded_to_64():
    import torch
    from paper_1701_04900_gb300.batch import MultiLaneSolver
    d = nesterov_lasso(600, 2000, 20, lam=1.0, seed=71, store_dtype=np.float32)
    lams = list(np.geomspace(20.0, 1.0, 40))
    At, B = _lanes(d, [d["b"]] * 40, lams)
    ms = MultiLaneSolver(At, B, lams, d["m"], max_sweeps=3000, tol_stat=1e-6)
    X = torch.zeros((40, d["n"]), dtype=torch.float32, device="cuda")
    per, tot = ms.solve(X)
    assert tot["status"] == 0
    assert all(st["stat_xhat"] <= 1e-6 for st in per)
    for l in (0, 20, 39):
        q = O.Problem.from_data(d)
        q.lam = lams[l]
        xl = X[l].cpu().numpy().astype(np.float64)
        assert O.stationarity(O.xhat_merit(q, xl, O.surrogate_weights(q)), xl) <= 1.5e-6, l
    p = O.Problem.from_data(d)
    x = X[-1].cpu().numpy().astype(np.float64)
    f1 = O.objective(p, d["x_star"])
    assert (O.objective(p, x) - f1) / f1 <= 1e-5
    ms.close()


def test_multi_rejects_what_it_does_not_support():
    import torch
    from paper_1701_04900_gb300 import AsyflexaError
    from paper_1701_04900_gb300.batch import MultiLaneSolver
    d = random_lasso(100, 64, seed=3, store_dtype=np.float32)
    At, B = _lanes(d, [d["b"]] * 3, [0.1] * 3)
    with pytest.raises(AsyflexaError):
        MultiLaneSolver(At, B, [0.1, -1.0, 0.1], d["m"])       # negative lambda
    B65 = torch.zeros((65, At.shape[1]), dtype=torch.float32, device="cuda")
    with pytest.raises(AsyflexaError):
        MultiLaneSolver(At, B65, [0.1] * 65, d["m"])             # more than 64 lanes
