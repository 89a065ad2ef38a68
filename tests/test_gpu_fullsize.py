"""Full-size checks on the 20000 x 100000 FP32 planted LASSO in the bench's launch shape.

The oracle cannot run whole sweeps at this size in seconds, so it checks sampled outputs
it can compute one by one:
  * sync: the first two Jacobi sweeps from x = 0.  The oracle computes its own x^1 for
    every column (column chunks, FP64) and x^2 on a random sample of columns from its own
    x^1 (no oracle input comes from the GPU); tolerance 1e-5 normwise.
  * async: a solve to a 1e-6 relative gap.  The oracle evaluates F(x) exactly from the
    nonzero columns and the merit ||xhat(x) - x||_inf on all nonzero columns plus a random
    sample of the others.
"""

import numpy as np
import pytest

import oracle as O
from tests._gpu_helpers import rel_inf

pytestmark = pytest.mark.gpu

M, N, K, LAM = 20000, 100000, 1000, 1.0


@pytest.fixture(scope="module")
def inst():
    import torch
    from paper_1701_04900_gb300.build import build_library
    from inputs import nesterov_lasso_torch
    build_library()
    g = nesterov_lasso_torch(M, N, K, lam=LAM, seed=0, device="cuda")
    b64 = g["b"].double().cpu().numpy()
    yield g, b64
    del g
    torch.cuda.empty_cache()


def host_cols(At, idx):
    """FP64 host copy of the columns idx (as an m x len(idx) matrix)."""
    import torch
    idx_t = torch.as_tensor(np.asarray(idx), device="cuda", dtype=torch.long)
    return At[idx_t, :M].double().cpu().numpy().T


def oracle_jacobi_first_sweep(At, b64, dw, gamma, chunk=8192):
    """x^1 from x^0 = 0 for every column: g = A^T (A*0 - b)."""
    x1 = np.zeros(N)
    r0 = -b64
    for j0 in range(0, N, chunk):
        cols = np.arange(j0, min(N, j0 + chunk))
        Ac = host_cols(At, cols)
        g = Ac.T @ r0
        xh = O.best_response(np.zeros(cols.size), g, dw[cols], LAM, -np.inf, np.inf)
        x1[cols] = gamma * xh
    return x1


def test_fullsize_sync_two_sweeps_sampled(inst):
    import torch
    from paper_1701_04900_gb300 import Solver
    g, b64 = inst
    At = g["At"]
    gamma, tau_rel = 0.9, 4.0
    s = Solver(At, g["b"], LAM, m=M, block_w=32, mode="sync", gamma=gamma, tau_rel=tau_rel)
    dw = s.weights().cpu().numpy()
    # the weights themselves: kappa_j = ||a_j||^2 on a sample, FP64
    rng = np.random.default_rng(0)
    samp = np.sort(rng.choice(N, size=4096, replace=False))
    Asamp = host_cols(At, samp)
    want_dw = (1.0 + tau_rel) * np.einsum("ij,ij->j", Asamp, Asamp)
    assert rel_inf(dw[samp], want_dw) < 1e-12
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    s.step(x, 1)
    x1_gpu = x.cpu().numpy().astype(np.float64)
    x1 = oracle_jacobi_first_sweep(At, b64, weights_oracle(At, tau_rel), gamma)
    assert rel_inf(x1_gpu, x1) < 1e-5
    s.step(x, 1)
    x2_gpu = x.cpu().numpy().astype(np.float64)
    nz = np.nonzero(x1)[0]
    r1 = host_cols(At, nz) @ x1[nz] - b64
    g2 = Asamp.T @ r1
    dws = weights_oracle_cols(Asamp, tau_rel)
    x2 = x1[samp] + gamma * (O.best_response(x1[samp], g2, dws, LAM, -np.inf, np.inf) - x1[samp])
    assert rel_inf(x2_gpu[samp], x2) < 1e-5
    s.close()


def weights_oracle_cols(Acols, tau_rel):
    return (1.0 + tau_rel) * np.einsum("ij,ij->j", Acols, Acols)


def weights_oracle(At, tau_rel, chunk=8192):
    out = np.zeros(N)
    for j0 in range(0, N, chunk):
        cols = np.arange(j0, min(N, j0 + chunk))
        out[cols] = weights_oracle_cols(host_cols(At, cols), tau_rel)
    return out


def test_fullsize_async_solve_reaches_gap(inst):
    import torch
    from paper_1701_04900_gb300 import Solver
    g, b64 = inst
    At = g["At"]
    sup = g["support"].cpu().numpy()
    xs = g["x_star"].cpu().numpy()
    r_star = host_cols(At, sup) @ xs[sup] - b64
    f_ref = 0.5 * float(r_star @ r_star) + LAM * float(np.abs(xs).sum())
    s = Solver(At, g["b"], LAM, m=M, block_w=32, mode="async", gamma=0.9, refresh_every=10, check_every=10,
               max_sweeps=3000, f_star=f_ref)
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    st = s.solve(x)
    assert st["status"] == 0, st
    xg = x.cpu().numpy().astype(np.float64)
    nz = np.nonzero(xg)[0]
    Anz = host_cols(At, nz)
    r = Anz @ xg[nz] - b64
    F = 0.5 * float(r @ r) + LAM * float(np.abs(xg).sum())
    assert (F - f_ref) / f_ref <= 1.5e-6
    assert abs(F - st["F"]) <= 1e-9 * F
    rng = np.random.default_rng(1)
    others = rng.choice(N, size=8192, replace=False)
    cols = np.union1d(nz, others)
    Ac = host_cols(At, cols)
    gcol = Ac.T @ r
    dcol = np.einsum("ij,ij->j", Ac, Ac)
    merit = O.best_response(xg[cols], gcol, dcol, LAM, -np.inf, np.inf) - xg[cols]
    assert O.stationarity(merit, xg) <= 1.5e-6
    s.close()
