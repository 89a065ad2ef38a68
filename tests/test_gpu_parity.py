"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (normwise relative, ||x_gpu - x_oracle||_inf / ||x_oracle||_inf):
  FP64 storage: 1e-10;  FP32 / BF16 / FP8 storage (FP32 arithmetic): 1e-5.
The oracle sees exactly the stored values (FP32 / dequantised codes widened to FP64).
"""

import math

import numpy as np
import pytest

import oracle as O
from inputs import dc_problem, nesterov_lasso, random_lasso, ncquad_problem
from tests._gpu_helpers import quantize_columns, rel_inf, to_cuda

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1701_04900_gb300.build import build_library
    assert torch.cuda.is_available()
    build_library()


def make_solver(d, **kw):
    from paper_1701_04900_gb300 import Solver
    t = to_cuda(d)
    loss = kw.pop("loss", "lasso")
    c = kw.pop("c", d.get("c", 0.0))
    return Solver(t["At"], t["b"], d["lam"], m=d["m"], lo=t.get("lo"), hi=t.get("hi"), loss=loss, c=c, **kw)


def xzeros(d, dtype):
    import torch
    return torch.zeros(d["n"], dtype=dtype, device="cuda")


def oracle_jacobi(p, d_w, gamma, sweeps, x0=None):
    x = np.zeros(p.n) if x0 is None else x0.copy()
    r = O.residual(p, x)
    out = []
    for _ in range(sweeps):
        x, r = O.jacobi_sweep(p, x, r, d_w, gamma)
        out.append(x.copy())
    return out


# ----------------------------------------------------------------------------- create

@pytest.mark.parametrize("store", [np.float64, np.float32])
@pytest.mark.parametrize("loss", ["lasso", "ncquad"])
def test_weights_match_oracle(store, loss):
    if loss == "lasso":
        d = random_lasso(301, 257, seed=1, store_dtype=store)
        p = O.Problem.from_data(d)
    else:
        d = ncquad_problem(400, 300, seed=1, store_dtype=store)
        p = O.Problem.from_data(d, loss="ncquad")
    s = make_solver(d, loss=loss, tau=0.25, tau_rel=0.5)
    got = s.weights().cpu().numpy()
    want = O.surrogate_weights(p, tau=0.25, tau_rel=0.5)
    assert rel_inf(got, want) < 1e-13


@pytest.mark.parametrize("store", [np.float64, np.float32])
def test_refresh_matches_oracle_residual(store):
    import torch
    d = random_lasso(1003, 777, seed=2, store_dtype=store)
    p = O.Problem.from_data(d)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(777) * (rng.random(777) < 0.3)
    x = x.astype(store)
    s = make_solver(d)
    xt = torch.from_numpy(x).cuda()
    s.refresh(xt)
    got = s.residual().cpu().numpy()
    want = O.residual(p, x.astype(np.float64))
    assert rel_inf(got, want) < 1e-14


# ----------------------------------------------------------------------------- sync Jacobi

def run_sync_parity(d, w, gamma, sweeps_list, tol, store, loss="lasso", tau=0.0, use_safe=True, num_ctas=0):
    import torch
    p = O.Problem.from_data(d, loss=loss)
    tr = O.jacobi_tau_rel(p, gamma) if use_safe else 0.0
    dw = O.surrogate_weights(p, tau=tau, tau_rel=tr)
    ref = oracle_jacobi(p, dw, gamma, max(sweeps_list))
    s = make_solver(d, loss=loss, block_w=w, mode="sync", gamma=gamma, tau=tau, tau_rel=tr, num_ctas=num_ctas)
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    done = 0
    worst = 0.0
    for k in sweeps_list:
        s.step(x, k - done)
        done = k
        e = rel_inf(x.cpu().numpy(), ref[k - 1])
        worst = max(worst, e)
        assert e < tol, (k, e)
    return worst


def test_sync_parity_config1_fp64():
    """LASSO FP64 200 x 1000, Nesterov planted (50 nonzeros), scalar blocks, gamma = 0.9."""
    d = nesterov_lasso(200, 1000, 50, lam=1.0, seed=0)
    run_sync_parity(d, 1, 0.9, [1, 5, 20, 60], TOL64, np.float64)


def test_sync_parity_fp32_slice():
    d = nesterov_lasso(2000, 10000, 100, lam=1.0, seed=1, store_dtype=np.float32)
    run_sync_parity(d, 32, 0.9, [1, 3, 10], TOL32, np.float32)


@pytest.mark.parametrize("store,tol", [(np.float64, TOL64), (np.float32, TOL32)])
def test_sync_parity_ragged_with_box(store, tol):
    d = random_lasso(1003, 777, seed=3, lam=0.05, store_dtype=store, zero_cols=3, box=0.5)
    run_sync_parity(d, 32, 0.9, [1, 4, 12], tol, store, tau=0.1)


@pytest.mark.parametrize("store,tol", [(np.float64, TOL64), (np.float32, TOL32)])
def test_sync_parity_ncquad(store, tol):
    d = ncquad_problem(300, 500, seed=4, store_dtype=store)
    run_sync_parity(d, 16, 0.9, [1, 5, 15], tol, store, loss="ncquad")


def test_sync_parity_grid_independent():
    """The Jacobi result does not depend on the number of CTAs (fixed reduction order)."""
    import torch
    d = nesterov_lasso(500, 3000, 30, seed=5, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    tr = O.jacobi_tau_rel(p, 0.9)
    xs = []
    for ctas in (1, 7, 0):
        s = make_solver(d, block_w=32, mode="sync", tau_rel=tr, num_ctas=ctas)
        x = xzeros(d, torch.float32)
        s.step(x, 6)
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[0], xs[2])


def test_sync_bitwise_reproducible():
    import torch
    d = nesterov_lasso(2000, 10000, 100, seed=6, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    tr = O.jacobi_tau_rel(p, 0.9)
    outs = []
    for _ in range(2):
        s = make_solver(d, block_w=32, mode="sync", tau_rel=tr)
        x = xzeros(d, torch.float32)
        s.step(x, 8)
        outs.append((x.cpu().numpy(), s.residual().cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_sync_multitile_residual():
    """m larger than one shared-memory residual tile (several tiles per panel)."""
    d = random_lasso(60001, 96, seed=7, lam=0.5, dist="gauss", store_dtype=np.float32)
    run_sync_parity(d, 8, 0.9, [1, 3], TOL32, np.float32)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_sync_parity_quantized_storage(kind):
    import torch
    from paper_1701_04900_gb300 import Solver
    d = random_lasso(1000, 800, seed=8, lam=0.02, dist="gauss", store_dtype=np.float32)
    q, scale, deq = quantize_columns(d["At"], d["m"], kind)
    p = O.Problem(A=deq.T, b=d["b"].astype(np.float64), lam=d["lam"])
    gamma = 0.9
    tr = O.jacobi_tau_rel(p, gamma)
    dw = O.surrogate_weights(p, tau_rel=tr)
    ref = oracle_jacobi(p, dw, gamma, 6)
    b = torch.from_numpy(d["b"]).cuda()
    s = Solver(q, b, d["lam"], m=d["m"], col_scale=scale, block_w=32, mode="sync", tau_rel=tr)
    assert rel_inf(s.weights().cpu().numpy(), dw) < 1e-12
    x = torch.zeros(d["n"], dtype=torch.float32, device="cuda")
    s.step(x, 6)
    assert rel_inf(x.cpu().numpy(), ref[-1]) < TOL32


# ----------------------------------------------------------------------------- async

@pytest.mark.parametrize("store,tol,variant", [(np.float64, TOL64, 0), (np.float32, TOL32, 1),
                                               (np.float32, TOL32, 2), (np.float32, TOL32, 3)])
@pytest.mark.parametrize("w", [1, 4, 32])
def test_async_single_cta_equals_gauss_seidel(store, tol, variant, w):
    """One CTA owns every block and runs them in order: exactly cyclic block Gauss-Seidel.
    variant 1 = staged-residual kernel, 2 = register-increment kernel with the column held in
    registers, 3 = register-increment kernel with a producer warp."""
    import torch
    d = random_lasso(301, 200, seed=9, lam=0.3, store_dtype=store, box=0.8)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=0.2)
    x_ref = np.zeros(p.n)
    r_ref = O.residual(p, x_ref)
    s = make_solver(d, block_w=w, mode="async", tau=0.2, num_ctas=1, refresh_every=100, variant=variant)
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    for sweep in range(3):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=w)
        s.step(x, 1)
        assert rel_inf(x.cpu().numpy(), x_ref) < tol, sweep


@pytest.mark.parametrize("m", [1021, 5003, 8192, 9001, 16384, 17001, 20477, 24571])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_async_single_cta_shapes(m, variant):
    """Column lengths spanning 1..6 shared-memory stages of the register kernels (ragged last
    unit included; 8192 and 16384 fill every stage, so no stage takes the checked path),
    against Gauss-Seidel."""
    import torch
    d = random_lasso(m, 48, seed=m, lam=0.2, dist="gauss", store_dtype=np.float32, box=2.0)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=0.05)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    for _ in range(2):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=8)
    s = make_solver(d, block_w=8, mode="async", tau=0.05, num_ctas=1, variant=variant)
    x = xzeros(d, torch.float32)
    s.step(x, 2)
    assert rel_inf(x.cpu().numpy(), x_ref) < TOL32


@pytest.mark.parametrize("m,n", [(2000, 600), (9001, 200), (10000, 96), (4000, 12000)])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_async_single_cta_ncquad_box_equals_gauss_seidel(m, n, variant):
    """Nonconvex quadratic with the box |x| <= 1 (gradient 2A^T r - 2c x, curvature
    2||a_j||^2 - 2c + tau), one CTA, against the oracle's cyclic Gauss-Seidel sweeps; long
    columns (several stages) and many blocks (large n) both covered."""
    import torch
    d = ncquad_problem(m, n, seed=m + n, store_dtype=np.float32)
    p = O.Problem.from_data(d, loss="ncquad")
    dw = O.surrogate_weights(p, tau=0.3)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    s = make_solver(d, block_w=32, mode="async", tau=0.3, num_ctas=1, refresh_every=100, variant=variant,
                    loss="ncquad")
    x = xzeros(d, torch.float32)
    for sweep in range(3):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=32)
        s.step(x, 1)
        assert rel_inf(x.cpu().numpy(), x_ref) < TOL32, sweep


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_async_single_cta_quantized(kind, variant):
    _single_cta_quantized(kind, variant, 3001)


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("m", [16385, 20000, 24576])
def test_async_single_cta_fp8_two_stage_columns(m, variant):
    """FP8 columns of 16385..24576 rows span 2 shared-memory stages but need only 3 units per
    thread: the register kernel's partial-unit instance, against Gauss-Seidel."""
    _single_cta_quantized("fp8", variant, m, n=96)


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("m", [16385, 20480])
def test_async_single_cta_bf16_three_stage_columns(m, variant):
    """BF16 columns of 16385..20480 rows span 3 stages but need only 5 of their 6 units per
    thread: the 5-unit instance, against Gauss-Seidel."""
    _single_cta_quantized("bf16", variant, m, n=96)


def _single_cta_quantized(kind, variant, m, n=300):
    import torch
    from paper_1701_04900_gb300 import Solver
    d = random_lasso(m, n, seed=17, lam=0.02, dist="gauss", store_dtype=np.float32)
    q, scale, deq = quantize_columns(d["At"], d["m"], kind)
    p = O.Problem(A=deq.T, b=d["b"].astype(np.float64), lam=d["lam"])
    dw = O.surrogate_weights(p, tau=0.1)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    for _ in range(3):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=16)
    b = torch.from_numpy(d["b"]).cuda()
    s = Solver(q, b, d["lam"], m=d["m"], col_scale=scale, block_w=16, mode="async", tau=0.1, num_ctas=1,
               variant=variant)
    x = torch.zeros(d["n"], dtype=torch.float32, device="cuda")
    s.step(x, 3)
    assert rel_inf(x.cpu().numpy(), x_ref) < TOL32


def test_async_single_cta_multitile_equals_gauss_seidel():
    import torch
    d = random_lasso(50001, 40, seed=10, lam=0.5, dist="gauss", store_dtype=np.float32)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p)
    x_ref, r_ref = O.gauss_seidel_sweep(p, np.zeros(p.n), O.residual(p, np.zeros(p.n)), dw, 0.9, w=8)
    x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=8)
    s = make_solver(d, block_w=8, mode="async", num_ctas=1)
    x = xzeros(d, torch.float32)
    s.step(x, 2)
    assert rel_inf(x.cpu().numpy(), x_ref) < TOL32


@pytest.mark.parametrize("store,variant", [(np.float64, 0), (np.float32, 1), (np.float32, 2), (np.float32, 3)])
def test_async_reaches_planted_optimum(store, variant):
    """Many CTAs, stale reads: objective within 1e-6 of the optimum, stationarity <= 1e-6.

    16 CTAs x 32 columns keep ~5% of the variables in flight, as in the 20000 x 100000
    bench configuration (152 CTAs x 32 of 100000)."""
    import torch
    d = nesterov_lasso(2000, 10000, 100, lam=1.0, seed=11, store_dtype=store)
    p = O.Problem.from_data(d)
    f_ref = O.objective(p, d["x_star"])   # optimal value on the stored data (up to ~1e-12)
    s = make_solver(d, block_w=32, mode="async", gamma=0.9, f_star=f_ref, max_sweeps=3000,
                    check_every=10, refresh_every=5, num_ctas=16, variant=variant)
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    st = s.solve(x)
    assert st["status"] == 0, st
    assert st["rel_gap"] <= 1e-6 and st["stat_xhat"] <= 1e-6
    xg = x.cpu().numpy().astype(np.float64)
    F = O.objective(p, xg)
    assert (F - f_ref) / f_ref <= 1.5e-6
    assert abs(F - st["F"]) <= 1e-9 * abs(F)
    dwt = O.surrogate_weights(p)
    assert O.stationarity(O.xhat_merit(p, xg, dwt), xg) <= 1.5e-6
    assert st["block_updates"] == st["sweeps"] * math.ceil(d["n"] / 32)
    assert sum(st["staleness_hist"]) == st["block_updates"]


def test_check_measures_match_oracle():
    import torch
    d = random_lasso(777, 501, seed=12, lam=0.4, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(p.n) * (rng.random(p.n) < 0.2)).astype(np.float32)
    s = make_solver(d, tau=0.3)
    st = s.check(torch.from_numpy(x).cuda())
    x64 = x.astype(np.float64)
    assert abs(st["F"] - O.objective(p, x64)) <= 1e-12 * abs(O.objective(p, x64))
    assert abs(st["stat_mf"] - O.stationarity(O.mf_measure(p, x64), x64)) <= 1e-9
    dwt = O.surrogate_weights(p, tau=0.3)
    assert abs(st["stat_xhat"] - O.stationarity(O.xhat_merit(p, x64, dwt), x64)) <= 1e-9
    assert abs(st["kkt_viol"] - O.kkt_violation(p, x64)) <= 1e-9
    assert st["nnz"] == int(np.count_nonzero(x))


# ----------------------------------------------------------------------------- edge cases

def test_degenerate_shapes_and_bounds():
    import torch
    # n = 1, m = 1
    d = random_lasso(1, 1, seed=13, lam=0.1)
    p = O.Problem.from_data(d)
    s = make_solver(d, block_w=32, mode="async")
    x = xzeros(d, torch.float64)
    s.step(x, 3)
    xr = np.zeros(1)
    rr = O.residual(p, xr)
    for _ in range(3):
        xr, rr = O.gauss_seidel_sweep(p, xr, rr, O.surrogate_weights(p), 0.9, w=32)
    assert rel_inf(x.cpu().numpy(), xr) < TOL64
    # lo = hi: the best response is the bound; the fixed step moves a fraction gamma of
    # the way each sweep (gamma = 1 lands on it, gamma = 0.9 leaves 0.1^k of the distance)
    d = random_lasso(40, 30, seed=14, lam=0.1, box=1.0)
    d["lo"][:5] = 0.25
    d["hi"][:5] = 0.25
    for gamma, want in ((1.0, 0.25), (0.9, 0.25 * (1 - 0.1 ** 2))):
        s = make_solver(d, block_w=4, mode="sync", gamma=gamma)
        x = xzeros(d, torch.float64)
        s.step(x, 2)
        np.testing.assert_allclose(x.cpu().numpy()[:5], want, rtol=1e-15)
    # more columns per block than columns in the problem
    d = random_lasso(17, 5, seed=16, lam=0.05)
    p = O.Problem.from_data(d)
    s = make_solver(d, block_w=32, mode="sync")
    x = xzeros(d, torch.float64)
    s.step(x, 3)
    ref = oracle_jacobi(p, O.surrogate_weights(p), 0.9, 3)
    assert rel_inf(x.cpu().numpy(), ref[-1]) < TOL64


def test_async_delay_knob_widens_staleness_and_the_solve_still_converges():
    """The test-only delay (opts.delay_ns, a bounded staleness injection): odd CTAs sleep 500 us
    before each scatter, so their updates complete after many more of the others'.  The
    longest delays the staleness histogram holds (the largest log2 bucket with at least 1 % of
    the updates) grow by at least 4x, and the solve still reaches the gap and the stationarity
    the oracle confirms; out-of-range values are EINVAL."""
    import torch
    from paper_1701_04900_gb300.native import AsyflexaError
    d = nesterov_lasso(4000, 8000, 80, lam=1.0, seed=21, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    f_ref = O.objective(p, d["x_star"])
    tails = []
    for delay in (0, 500000):
        s = make_solver(d, block_w=32, mode="async", num_ctas=16, max_sweeps=3000, f_star=f_ref, delay_ns=delay)
        x = xzeros(d, torch.float32)
        st = s.solve(x)
        assert st["status"] == 0, (delay, st)
        xg = x.cpu().numpy().astype(np.float64)
        assert (O.objective(p, xg) - f_ref) / f_ref <= 1.5e-6
        assert O.stationarity(O.xhat_merit(p, xg, O.surrogate_weights(p)), xg) <= 1.5e-6
        h = np.array(st["staleness_hist"], dtype=np.float64)
        tails.append(int(np.nonzero(h >= 0.01 * h.sum())[0].max()))
    assert tails[1] >= tails[0] + 2, tails
    for bad in (-1, 1000001):
        with pytest.raises(AsyflexaError):
            make_solver(d, block_w=32, mode="async", delay_ns=bad)


@pytest.mark.parametrize("store", [np.float64, np.float32])
def test_async_divergence_is_reported(store):
    """A step that overshoots by construction: 64 x 4096 with nearly identical columns (all
    ones plus 1e-3 U[-1, 1]) and blocks of 8 columns.  The 8 columns of a block see the same
    residual and each one alone would remove its whole projection, so even one block update
    multiplies that part of r by about 1 - 8 * 0.9 = -6.2 (the FP64 oracle's Jacobi sweep grows
    ||r||_inf by about 3e3 per sweep).  The iterates overflow within the first check interval,
    and the library must report ENONFINITE instead of returning a number."""
    import torch
    from paper_1701_04900_gb300 import AsyflexaError
    rng = np.random.default_rng(4)
    m, n = 64, 4096
    A = (1.0 + 1e-3 * rng.uniform(-1, 1, (m, n))).astype(store)
    d = dict(At=np.ascontiguousarray(A.T), b=rng.standard_normal(m).astype(store), lam=1e-3, m=m, n=n)
    s = make_solver(d, block_w=8, mode="async", gamma=0.9, max_sweeps=400, check_every=10)
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    with pytest.raises(AsyflexaError) as ei:
        s.solve(x)
    assert ei.value.code == -5
    s.close()


@pytest.mark.parametrize("store", [np.float64, np.float32])
def test_nan_in_b_is_reported(store):
    """Host-side fault injection: a NaN in b makes the residual, and with it F, non-finite.
    The solve must stop with ENONFINITE (no kernel faults or waits on the value)."""
    import torch
    from paper_1701_04900_gb300 import AsyflexaError
    d = random_lasso(300, 500, seed=21, lam=0.1, store_dtype=store)
    d["b"] = d["b"].copy()
    d["b"][17] = np.nan
    for mode in ("async", "sync"):
        s = make_solver(d, block_w=32, mode=mode, max_sweeps=50, check_every=5)
        x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
        with pytest.raises(AsyflexaError) as ei:
            s.solve(x)
        assert ei.value.code == -5
        s.close()


def test_invalid_inputs_are_rejected():
    import torch
    from paper_1701_04900_gb300 import AsyflexaError
    d = random_lasso(40, 30, seed=15, box=1.0)
    d["lo"][3] = 2.0     # lo > hi
    with pytest.raises(AsyflexaError) as ei:
        make_solver(d)
    assert ei.value.code == -1
    d = ncquad_problem(40, 30, seed=15)
    with pytest.raises(AsyflexaError) as ei:
        make_solver(d, loss="ncquad", c=1e6)      # negative surrogate weights
    assert ei.value.code == -1
    d = random_lasso(40, 30, seed=15)
    s = make_solver(d)
    with pytest.raises(ValueError):
        s.step(torch.zeros(30, dtype=torch.float32, device="cuda"), 1)


def test_kernel_variant_reports_the_form_launched():
    """Automatic choice on FP32 storage: the producer-warp form (3) up to 12288 rows, the
    column-in-registers form (2) above; variants 2 and 3 force a form; the compensated
    gradient runs the producer-warp form; variant 1 and FP64 storage: the staged kernel (1)."""
    d = random_lasso(5000, 64, seed=17, store_dtype=np.float32)
    for kw, want in (({}, 3), ({"variant": 2}, 2), ({"variant": 3}, 3), ({"variant": 2, "exact_grad": 1}, 3),
                     ({"variant": 1}, 1)):
        s = make_solver(d, mode="async", **kw)
        assert s.read_counters()["kernel_variant"] == want, kw
        s.close()
    d = random_lasso(12289, 40, seed=18, store_dtype=np.float32)
    for kw, want in (({}, 2), ({"variant": 3}, 3)):
        s = make_solver(d, mode="async", **kw)
        assert s.read_counters()["kernel_variant"] == want, kw
        s.close()
    s = make_solver(random_lasso(300, 16, seed=16, store_dtype=np.float64), mode="async")
    assert s.read_counters()["kernel_variant"] == 1
    s.close()


def test_unsupported_kernel_variant_is_reported():
    """A requested kernel that does not cover the problem is refused at create (no fallback)."""
    from paper_1701_04900_gb300 import AsyflexaError
    d = random_lasso(24581, 16, seed=16, store_dtype=np.float32)
    for v in (2, 3):
        with pytest.raises(AsyflexaError) as ei:
            make_solver(d, mode="async", variant=v)
        assert ei.value.code == -6
    d = random_lasso(300, 16, seed=16, store_dtype=np.float64)
    for v in (2, 3):
        with pytest.raises(AsyflexaError) as ei:
            make_solver(d, mode="async", variant=v)
        assert ei.value.code == -6


# ----------------------------------------------------------------------------- DC regularisers

@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("m,n", [(700, 500), (9001, 160)])
def test_async_single_cta_dc_equals_gauss_seidel(reg, variant, m, n):
    """F = ||Ax-b||^2 + lam H(x) (Section 4.3) with the log / exp regulariser: one CTA against
    the oracle's cyclic Gauss-Seidel sweeps (concave part linearised at each block's x)."""
    import torch
    d = dc_problem(m, n, reg=reg[3:], seed=m + n, store_dtype=np.float32)
    p = O.Problem.from_data(d, loss=reg)
    dw = O.surrogate_weights(p, tau=0.1)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    s = make_solver(d, block_w=32, mode="async", tau=0.1, num_ctas=1, refresh_every=100, variant=variant,
                    loss=reg, theta=d["theta"])
    x = xzeros(d, torch.float32)
    for sweep in range(4):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=32)
        s.step(x, 1)
        assert rel_inf(x.cpu().numpy(), x_ref) < TOL32, sweep


@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
@pytest.mark.parametrize("store,tol", [(np.float64, TOL64), (np.float32, TOL32)])
def test_sync_parity_dc(reg, store, tol):
    d = dc_problem(400, 600, reg=reg[3:], seed=8, store_dtype=store)
    import torch
    p = O.Problem.from_data(d, loss=reg)
    dw = O.surrogate_weights(p, tau_rel=1.0)
    ref = oracle_jacobi(p, dw, 0.9, 12)
    s = make_solver(d, block_w=16, mode="sync", gamma=0.9, tau_rel=1.0, loss=reg, theta=d["theta"])
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    done = 0
    for k in (1, 4, 12):
        s.step(x, k - done)
        done = k
        assert rel_inf(x.cpu().numpy(), ref[k - 1]) < tol, k


@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
def test_dc_async_reaches_a_stationary_point(reg):
    """Many CTAs: the solve stops at ||xhat(x) - x||_inf / max(1, ||x||_inf) <= 1e-6 measured by
    the library; the oracle confirms the stationarity and the objective at the returned x."""
    import torch
    d = dc_problem(2000, 4000, reg=reg[3:], seed=9, store_dtype=np.float32)
    p = O.Problem.from_data(d, loss=reg)
    s = make_solver(d, block_w=32, mode="async", num_ctas=16, max_sweeps=3000, check_every=10, refresh_every=10,
                    tol_stat=1e-6, loss=reg, theta=d["theta"])
    x = xzeros(d, torch.float32)
    st = s.solve(x)
    assert st["status"] == 0, st
    xr = x.cpu().numpy().astype(np.float64)
    merit = O.stationarity(O.xhat_merit(p, xr, O.surrogate_weights(p)), xr)
    assert merit <= 2e-6
    assert abs(O.objective(p, xr) - st["F"]) <= 1e-9 * abs(st["F"])
    assert abs(st["stat_xhat"] - merit) <= 1e-7


@pytest.mark.parametrize("reg", ["dc_log", "dc_exp"])
def test_dc_check_measures_match_oracle(reg):
    import torch
    d = dc_problem(1500, 900, reg=reg[3:], seed=10, store_dtype=np.float64)
    p = O.Problem.from_data(d, loss=reg)
    rng = np.random.default_rng(1)
    xv = rng.standard_normal(p.n) * (rng.random(p.n) < 0.2)
    s = make_solver(d, tau=0.2, loss=reg, theta=d["theta"])
    xt = torch.from_numpy(xv).cuda()
    s.refresh(xt)
    st = s.check(xt)
    dw = O.surrogate_weights(p, tau=0.2)
    assert st["F"] == pytest.approx(O.objective(p, xv), rel=1e-12)
    assert st["stat_xhat"] == pytest.approx(O.stationarity(O.xhat_merit(p, xv, dw), xv), rel=1e-9)
    assert st["stat_mf"] == pytest.approx(O.stationarity(O.mf_measure(p, xv), xv), rel=1e-9)


# ----------------------------------------------------------------------------- diminishing step

@pytest.mark.parametrize("store,tol,variant", [(np.float64, TOL64, 0), (np.float32, TOL32, 1),
                                               (np.float32, TOL32, 2), (np.float32, TOL32, 3)])
def test_async_single_cta_diminishing_step_equals_gauss_seidel(store, tol, variant):
    """gamma^{k+1} = gamma^k (1 - mu gamma^k) (the experiments' rule, Section 4) with k counting
    block updates: one CTA performs them in order, so update k of the run takes gamma^k."""
    import torch
    d = random_lasso(1201, 300, seed=21, lam=0.2, store_dtype=store, box=1.5)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=0.1)
    w = 16
    N = len(O.block_ranges(p.n, w))
    steps = O.diminishing_steps(1.0, 0.02, 5 * N)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    s = make_solver(d, block_w=w, mode="async", tau=0.1, gamma=1.0, gamma_mu=0.02, num_ctas=1, refresh_every=3,
                    variant=variant)
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    for sweep in range(5):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, steps[sweep * N:(sweep + 1) * N], w=w)
        s.step(x, 1)
        assert rel_inf(x.cpu().numpy(), x_ref) < tol, sweep
    assert steps[-1] < 0.5     # the sequence did diminish over the run


@pytest.mark.parametrize("store,tol", [(np.float64, TOL64), (np.float32, TOL32)])
def test_sync_diminishing_step_parity(store, tol):
    """Jacobi sweeps: block i of sweep s is update s N + i of the sequence."""
    import torch
    d = nesterov_lasso(300, 1200, 20, seed=22, store_dtype=store)
    p = O.Problem.from_data(d)
    w = 32
    N = len(O.block_ranges(p.n, w))
    tr = O.jacobi_tau_rel(p, 1.0)
    dw = O.surrogate_weights(p, tau_rel=tr)
    steps = O.diminishing_steps(1.0, 0.01, 8 * N)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    s = make_solver(d, block_w=w, mode="sync", gamma=1.0, gamma_mu=0.01, tau_rel=tr)
    x = xzeros(d, torch.float64 if store == np.float64 else torch.float32)
    for sweep in range(8):
        x_ref, r_ref = O.jacobi_sweep(p, x_ref, r_ref, dw, O.block_steps(p.n, w, steps[sweep * N:(sweep + 1) * N]))
    s.step(x, 8)
    assert rel_inf(x.cpu().numpy(), x_ref) < tol


def test_diminishing_step_solve_restarts_the_sequence():
    """Every solve runs the sequence from gamma^0: two Jacobi solves from x = 0 agree bitwise."""
    import torch
    d = nesterov_lasso(300, 1200, 20, seed=23, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    s = make_solver(d, block_w=32, mode="sync", gamma=1.0, gamma_mu=1e-3, tau_rel=O.jacobi_tau_rel(p, 1.0),
                    max_sweeps=40, check_every=10, tol_stat=0.0)
    xs = []
    for _ in range(2):
        x = xzeros(d, torch.float32)
        s.solve(x)
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


# ------------------------------------------------------------- duality-gap certificate (LASSO)

def test_dual_gap_certificate_matches_oracle():
    import torch
    d = random_lasso(900, 700, seed=24, lam=0.4, dist="gauss")
    p = O.Problem.from_data(d)
    rng = np.random.default_rng(3)
    xv = rng.standard_normal(p.n) * (rng.random(p.n) < 0.1) * 0.1
    s = make_solver(d)
    xt = torch.from_numpy(xv).cuda()
    s.refresh(xt)
    st = s.check(xt)
    P, gap = O.lasso_dual_gap(p, xv)
    assert st["F"] == pytest.approx(P, rel=1e-12)
    assert st["dual_gap"] == pytest.approx(gap / max(1.0, abs(P)), rel=1e-9)


def test_liu_wright_solve_reaches_the_oracle_optimum():
    """The Gaussian LASSO set of Section 4.2 (no closed-form optimum): the async solve stops at
    stationarity <= 1e-6; the oracle's Gauss-Seidel optimum confirms a relative gap <= 1e-6,
    and the reported duality-gap certificate agrees with the oracle's at the returned x."""
    import torch
    from inputs import liu_wright_lasso
    d = liu_wright_lasso(1500, 3000, 15, seed=25, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    s = make_solver(d, block_w=32, mode="async", num_ctas=8, max_sweeps=3000, check_every=10, refresh_every=10,
                    tol_stat=1e-6)
    x = xzeros(d, torch.float32)
    st = s.solve(x)
    assert st["status"] == 0, st
    _, F_or, _ = O.solve_gs(p, w=32, gamma=1.0, max_sweeps=2000, tol=1e-15)
    xr = x.cpu().numpy().astype(np.float64)
    F = O.objective(p, xr)
    assert (F - F_or) / F_or <= 1e-6
    P, gap = O.lasso_dual_gap(p, xr)
    assert st["dual_gap"] == pytest.approx(gap / max(1.0, abs(P)), rel=1e-6, abs=1e-12)


# ---------------------------------------------------------------- adaptive proximal weight

def test_adaptive_tau_recovers_an_unstable_async_run():
    """Every block of a small problem in flight at once with no proximal weight is the setting
    that can diverge (test above); with tau_adapt the solve raises tau whenever a check
    interval raised F, and reaches the planted optimum."""
    import torch
    d = nesterov_lasso(2000, 10000, 100, lam=1.0, seed=11, store_dtype=np.float64)
    p = O.Problem.from_data(d)
    f_ref = O.objective(p, d["x_star"])
    s = make_solver(d, block_w=32, mode="async", gamma=0.9, max_sweeps=3000, check_every=1, refresh_every=1,
                    tau_adapt=True, f_star=f_ref, tol_stat=1e-6)
    x = xzeros(d, torch.float64)
    st = s.solve(x)
    assert st["status"] == 0, st
    assert st["rel_gap"] <= 1e-6
    assert O.objective(p, x.cpu().numpy()) == pytest.approx(st["F"], rel=1e-12)


def test_adaptive_tau_leaves_a_descent_run_unchanged():
    """One CTA is cyclic Gauss-Seidel, whose LASSO objective never rises: tau stays 0 and the
    iterates are the oracle's."""
    import torch
    d = random_lasso(600, 300, seed=26, lam=0.3, store_dtype=np.float64)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    for _ in range(30):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=16)
    s = make_solver(d, block_w=16, mode="async", gamma=0.9, num_ctas=1, max_sweeps=30, check_every=1,
                    tau_adapt=True, tol_stat=0.0)
    x = xzeros(d, torch.float64)
    st = s.solve(x)
    assert st["tau_extra"] == 0.0
    assert rel_inf(x.cpu().numpy(), x_ref) < TOL64


# ----------------------------------------------------------------------------- compensated gradient

@pytest.mark.parametrize("m,w", [(301, 1), (301, 32), (17001, 8), (20477, 32)])
def test_async_single_cta_exact_grad_equals_gauss_seidel(m, w):
    """exact_grad = 1 (Dot2 accumulation of a_j^T r~): one CTA is still cyclic Gauss-Seidel, now
    within 2e-6 of the FP64 oracle (the FP32 snapshot of r and the FP32 x remain)."""
    import torch
    d = random_lasso(m, 64, seed=m + w, lam=0.3, dist="gauss", store_dtype=np.float32, box=0.8)
    p = O.Problem.from_data(d)
    dw = O.surrogate_weights(p, tau=0.2)
    x_ref, r_ref = np.zeros(p.n), O.residual(p, np.zeros(p.n))
    s = make_solver(d, block_w=w, mode="async", tau=0.2, num_ctas=1, refresh_every=100, variant=2, exact_grad=1)
    x = xzeros(d, torch.float32)
    for sweep in range(3):
        x_ref, r_ref = O.gauss_seidel_sweep(p, x_ref, r_ref, dw, 0.9, w=w)
        s.step(x, 1)
        assert rel_inf(x.cpu().numpy(), x_ref) < 2e-6, sweep


def test_exact_grad_option_is_validated():
    from paper_1701_04900_gb300 import AsyflexaError
    d32 = random_lasso(300, 16, seed=3, store_dtype=np.float32)
    d64 = random_lasso(300, 16, seed=3, store_dtype=np.float64)
    for d, kw in ((d64, {"mode": "async"}), (d32, {"mode": "sync"}), (d32, {"mode": "async", "variant": 1})):
        with pytest.raises(AsyflexaError) as ei:
            make_solver(d, exact_grad=1, **kw)
        assert ei.value.code == -6, kw
    with pytest.raises(AsyflexaError) as ei:
        make_solver(d32, mode="async", exact_grad=2)
    assert ei.value.code == -1


@pytest.mark.parametrize("known", [True, False])
@pytest.mark.parametrize("exact_grad", [0, 1])
def test_solve_stats_are_an_exact_check_of_the_result(known, exact_grad):
    """Whatever the check schedule, the solve stops on an exact check and returns its values:
    a separate check of the returned x gives the same F and stationarity, and both tolerances
    hold for the returned x against the oracle."""
    import torch
    d = nesterov_lasso(3000, 12000, 120, lam=1.0, seed=21, store_dtype=np.float32)
    p = O.Problem.from_data(d)
    f_ref = O.objective(p, d["x_star"])
    s = make_solver(d, block_w=32, mode="async", gamma=0.9, f_star=f_ref if known else math.nan,
                    tol_stat=1e-6, max_sweeps=3000, check_every=10, refresh_every=10, num_ctas=24, variant=2,
                    exact_grad=exact_grad)
    x = xzeros(d, torch.float32)
    st = s.solve(x)
    assert st["status"] == 0, st
    assert st["stat_xhat"] <= 1e-6
    chk = s.check(x)
    assert abs(chk["F"] - st["F"]) <= 1e-12 * abs(st["F"])
    assert abs(chk["stat_xhat"] - st["stat_xhat"]) <= 1e-9 * max(st["stat_xhat"], 1e-30) + 1e-15
    xg = x.cpu().numpy().astype(np.float64)
    assert O.stationarity(O.xhat_merit(p, xg, O.surrogate_weights(p)), xg) <= 1.5e-6
    if known:
        assert st["rel_gap"] <= 1e-6 and (O.objective(p, xg) - f_ref) / f_ref <= 1.5e-6


def test_handles_of_different_sizes_share_kernel_instances():
    """A kernel's shared-memory limit belongs to the kernel, not to a handle: a handle created
    after another one, for fewer rows, runs the same sweep-kernel instance with a smaller shared
    memory footprint, and must not leave the first handle unable to launch it.  Both handles
    solve (the older one first) to the gap and stationarity tolerances, confirmed at the
    returned x in FP64 against the planted optimum."""
    import torch
    from paper_1701_04900_gb300 import Solver
    from inputs import nesterov_lasso_torch
    n, lam = 3000, 1.0
    gens = [nesterov_lasso_torch(m, n, 30, lam=lam, seed=21 + i, device="cuda") for i, m in enumerate((20000, 18000))]
    f_refs, solvers = [], []
    for g, m in zip(gens, (20000, 18000)):
        A = g["At"][:, :m].double().T
        r = A @ g["x_star"].double() - g["b"].double()
        f_refs.append(0.5 * float(r @ r) + lam * float(g["x_star"].double().abs().sum()))
    for g, m, f in zip(gens, (20000, 18000), f_refs):
        solvers.append(Solver(g["At"], g["b"], lam, m=m, block_w=32, mode="async", gamma=0.9, max_sweeps=3000,
                              f_star=f))
    stats = []
    for g, m, f, s in zip(gens, (20000, 18000), f_refs, solvers):
        x = torch.zeros(n, dtype=torch.float32, device="cuda")
        st = s.solve(x)
        assert st["status"] == 0, st
        A = g["At"][:, :m].double().T
        xd = x.double()
        r = A @ xd - g["b"].double()
        F = 0.5 * float(r @ r) + lam * float(xd.abs().sum())
        assert (F - f) / f <= 1.5e-6
        gcol = (A.T @ r).cpu().numpy()
        dcol = (A * A).sum(0).cpu().numpy()
        xh = xd.cpu().numpy()
        merit = O.best_response(xh, gcol, dcol, lam, -np.inf, np.inf) - xh
        assert O.stationarity(merit, xh) <= 1.5e-6
        stats.append(st)
    assert stats[0]["kernel_variant"] == stats[1]["kernel_variant"]
    for s in solvers:
        s.close()
