"""asyflexa_residual_noalloc: the residual without a handle and without device allocation.

Callers that cannot allocate device memory at the point where they need r = A x - b (for
example a plugin that its host application gives a fixed device-memory budget, or a loop in
which cudaMalloc would synchronise the device) use this entry point.  The test calls it
through the C ABI twice in a row (the scratch array is shared and keeps the previous call's
contents) and compares each result with the existing handle entry point
asyflexa_residual_refresh + asyflexa_get_residual, for every storage type (BF16 and FP8 with
their per-column scales).  It lives in its own file, collected last, and needs no state from
other tests.
"""

import ctypes as C

import numpy as np
import pytest

from inputs import random_lasso

pytestmark = pytest.mark.gpu

TOL = 1e-12   # both sides accumulate exactly; only the grouping of partial sums differs


@pytest.mark.parametrize("store", ["f64", "f32", "bf16", "fp8"])
def test_noalloc_matches_handle_refresh_twice(store):
    import torch
    from paper_1701_04900_gb300 import Solver, native
    from paper_1701_04900_gb300.build import build_library
    from tests._gpu_helpers import quantize_columns
    build_library()
    L = native.lib()
    dt = np.float64 if store == "f64" else np.float32
    d = random_lasso(1003, 777, seed=21, lam=0.1, store_dtype=dt, zero_cols=2)
    b = torch.from_numpy(d["b"]).cuda()
    if store in ("bf16", "fp8"):
        At, scale, _ = quantize_columns(d["At"], d["m"], store)
        s = Solver(At, b, d["lam"], m=d["m"], col_scale=scale)
    else:
        At = torch.from_numpy(d["At"]).cuda()
        s = Solver(At, b, d["lam"], m=d["m"])
    rng = np.random.default_rng(5)
    store = dt
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = (rng.standard_normal(d["n"]) * (rng.random(d["n"]) < 0.4)).astype(store)
        xt = torch.from_numpy(x).cuda()
        s.refresh(xt)
        want = s.residual().cpu().numpy()
        out = torch.full((d["m"],), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.asyflexa_residual_noalloc(C.byref(s.problem), C.c_void_p(xt.data_ptr()),
                                         C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == native.OK, L.asyflexa_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= TOL, (call, err)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1701_04900_gb300 import native
    from paper_1701_04900_gb300.build import build_library
    build_library()
    L = native.lib()
    A = torch.zeros((4, 16), dtype=torch.float32, device="cuda")
    b = torch.zeros(16, dtype=torch.float32, device="cuda")
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    r = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = native.Problem()
    p.m, p.n, p.lda = 16, 4, 16
    p.a_dtype = p.x_dtype = native.F32
    p.A, p.b = A.data_ptr(), b.data_ptr()
    assert L.asyflexa_residual_noalloc(C.byref(p), C.c_void_p(x.data_ptr()), C.c_void_p(r.data_ptr()), None) == 0
    torch.cuda.synchronize()
    p.n = 300000                                   # columns beyond the limit (never read)
    assert L.asyflexa_residual_noalloc(C.byref(p), C.c_void_p(x.data_ptr()), C.c_void_p(r.data_ptr()),
                                       None) == native.EINVAL
    assert b"262144" in L.asyflexa_last_error(None)
    p.n, p.m, p.lda = 4, 700000, 700000            # rows beyond the limit (never read)
    assert L.asyflexa_residual_noalloc(C.byref(p), C.c_void_p(x.data_ptr()), C.c_void_p(r.data_ptr()),
                                       None) == native.EINVAL
    assert b"rows" in L.asyflexa_last_error(None)
