"""Host-side checks of the C ABI (no GPU needed, no compute calls).

* the library builds (or is built) and loads;
* it exports every function declared in include/asyflexa.h;
* the ctypes mirrors of the structs have the sizes and offsets gcc gives the header;
* argument validation that happens before any CUDA call returns EINVAL.
"""

import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "asyflexa.h")


@pytest.fixture(scope="module")
def L():
    from paper_1701_04900_gb300.build import build_library
    from paper_1701_04900_gb300 import native
    build_library()
    return native.lib()


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(asyflexa_[a-z_]+)\s*\(", src)))


def test_exports_every_header_function(L):
    from paper_1701_04900_gb300 import native
    names = header_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert sorted(native.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    for name in names:
        assert re.search(rf"\bT {name}$", out, flags=re.M), name


def test_struct_layout_matches_header(L):
    from paper_1701_04900_gb300 import native
    probe = r"""
#include <stdio.h>
#include <stddef.h>
#include "asyflexa.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("asyflexa_problem %zu\n", sizeof(asyflexa_problem));
  printf("asyflexa_opts %zu\n", sizeof(asyflexa_opts));
  printf("asyflexa_stats %zu\n", sizeof(asyflexa_stats));
  P(asyflexa_problem, lambda) P(asyflexa_problem, loss) P(asyflexa_problem, hi)
  P(asyflexa_opts, gamma) P(asyflexa_opts, num_ctas) P(asyflexa_opts, f_star) P(asyflexa_opts, seed)
  P(asyflexa_opts, switch_tol) P(asyflexa_opts, gamma_mu) P(asyflexa_opts, tau_adapt)
  P(asyflexa_opts, exact_grad) P(asyflexa_opts, delay_ns)
  P(asyflexa_stats, staleness_hist) P(asyflexa_stats, kernel_launches) P(asyflexa_stats, checked)
  P(asyflexa_stats, kernel_variant) P(asyflexa_stats, dual_gap) P(asyflexa_stats, tau_extra)
  P(asyflexa_stats, batch_form) P(asyflexa_stats, ctas_per_sm) P(asyflexa_stats, handed_over)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        cfile = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(cfile, "w").write(probe)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), cfile, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in lines if l)
    assert int(got["asyflexa_problem"]) == C.sizeof(native.Problem)
    assert int(got["asyflexa_opts"]) == C.sizeof(native.Opts)
    assert int(got["asyflexa_stats"]) == C.sizeof(native.Stats)
    mapping = {"asyflexa_problem": native.Problem, "asyflexa_opts": native.Opts, "asyflexa_stats": native.Stats}
    rename = {"lambda": "lam"}
    for k, v in got.items():
        if "." in k:
            t, f = k.split(".")
            assert getattr(mapping[t], rename.get(f, f)).offset == int(v), k


def test_defaults_and_status_strings(L):
    from paper_1701_04900_gb300 import native
    o = native.default_opts()
    assert o.block_w == 32 and o.mode == native.SYNC and o.gamma == 0.9
    assert o.refresh_every == 10 and o.max_sweeps == 1000
    assert o.f_star != o.f_star  # NaN
    assert o.gamma_mu == 0.0 and o.variant == 0
    assert L.asyflexa_version() == 1
    assert L.asyflexa_status_string(-1) == b"ASYFLEXA_EINVAL"
    assert L.asyflexa_status_string(1) == b"ASYFLEXA_ENOTCONV"


def test_null_arguments_rejected_without_gpu(L):
    from paper_1701_04900_gb300 import native
    h = C.c_void_p()
    assert L.asyflexa_create(None, None, None, None) == native.EINVAL
    assert L.asyflexa_create(C.byref(h), None, None, None) == native.EINVAL
    assert h.value is None
    p = native.Problem()
    o = native.default_opts()
    o.block_w = 0
    assert L.asyflexa_create(C.byref(h), C.byref(p), C.byref(o), None) == native.EINVAL
    assert b"block_w" in L.asyflexa_last_error(None)
    o = native.default_opts()
    p.m, p.n, p.lda = 10, 10, 10          # lda * 4 bytes not a multiple of 16
    p.a_dtype = p.x_dtype = native.F32
    p.A = 256
    p.b = 256
    assert L.asyflexa_create(C.byref(h), C.byref(p), C.byref(o), None) == native.EINVAL
    assert b"lda" in L.asyflexa_last_error(None)
    p.lda = 12
    p.A = 8                                # misaligned
    assert L.asyflexa_create(C.byref(h), C.byref(p), C.byref(o), None) == native.EINVAL
    assert L.asyflexa_step(None, None, 1) == native.EINVAL
    assert L.asyflexa_solve(None, None, None) == native.EINVAL
    assert L.asyflexa_destroy(None) == native.OK


def test_batch_multi_adjoint_noalloc_validation_without_gpu(L):
    """The batched, multi-lane, adjoint and no-allocation entry points check their arguments
    before any CUDA call: null pointers, out-of-range counts and sizes, unsupported storage and
    non-finite parameters come back as EINVAL or EUNSUPPORTED with a message, and nothing is
    created."""
    from paper_1701_04900_gb300 import native
    err = lambda: L.asyflexa_last_error(None)
    h = C.c_void_p()
    o = native.default_opts()
    p = native.Problem()
    p.m, p.n, p.lda = 64, 32, 64
    p.a_dtype = p.x_dtype = native.F32
    p.A = p.b = 256                       # never dereferenced: every call below fails first

    # batched
    assert L.asyflexa_batch_create(None, C.byref(p), 1, C.byref(o), 0, None) == native.EINVAL
    assert L.asyflexa_batch_create(C.byref(h), None, 1, C.byref(o), 0, None) == native.EINVAL
    assert h.value is None
    assert L.asyflexa_batch_create(C.byref(h), C.byref(p), 0, C.byref(o), 0, None) == native.EINVAL
    assert b"count" in err()
    o.block_w = 200
    assert L.asyflexa_batch_create(C.byref(h), C.byref(p), 1, C.byref(o), 0, None) == native.EINVAL
    assert b"block_w" in err() and h.value is None
    o = native.default_opts()
    assert L.asyflexa_batch_solve(None, None, None, None, None) == native.EINVAL
    assert L.asyflexa_batch_check(None, None, None, None) == native.EINVAL
    assert L.asyflexa_batch_destroy(None) == native.OK

    # multi-lane
    lam = (C.c_double * 65)(*([1.0] * 65))
    Bp = C.c_void_p(256)
    assert L.asyflexa_multi_create(None, C.byref(p), 2, Bp, 64, lam, C.byref(o), None) == native.EINVAL
    assert L.asyflexa_multi_create(C.byref(h), C.byref(p), 2, None, 64, lam, C.byref(o), None) == native.EINVAL
    for k in (0, 65):
        assert L.asyflexa_multi_create(C.byref(h), C.byref(p), k, Bp, 64, lam, C.byref(o), None) == native.EINVAL
        assert b"k must be" in err()
    p.a_dtype = native.BF16
    assert L.asyflexa_multi_create(C.byref(h), C.byref(p), 2, Bp, 64, lam, C.byref(o), None) == native.EUNSUPPORTED
    p.a_dtype = native.F32
    p.loss = native.LOSS_NCQUAD
    assert L.asyflexa_multi_create(C.byref(h), C.byref(p), 2, Bp, 64, lam, C.byref(o), None) == native.EUNSUPPORTED
    p.loss = native.LOSS_LASSO
    assert L.asyflexa_multi_create(C.byref(h), C.byref(p), 2, Bp, 63, lam, C.byref(o), None) == native.EINVAL
    assert b"ldb" in err()
    for bad in (-1.0, float("nan"), float("inf")):
        lam[1] = bad
        assert L.asyflexa_multi_create(C.byref(h), C.byref(p), 2, Bp, 64, lam, C.byref(o), None) == native.EINVAL
        assert b"lambda" in err()
    assert h.value is None
    assert L.asyflexa_multi_solve(None, None, 0, None, None, None) == native.EINVAL
    assert L.asyflexa_multi_destroy(None) == native.OK

    # adjoint
    d = C.c_double()
    A, x, v, db = C.c_void_p(256), C.c_void_p(512), C.c_void_p(768), C.c_void_p(1024)
    adj = lambda A_, lda, dt, m, n, tol: L.asyflexa_adjoint(A_, lda, dt, m, n, x, v, tol, None, C.byref(d), db,
                                                             None, None, None)
    assert adj(A, 64, native.BF16, 64, 32, 1e-6) == native.EUNSUPPORTED
    assert adj(None, 64, native.F32, 64, 32, 1e-6) == native.EINVAL
    assert adj(A, 64, native.F32, 0, 32, 1e-6) == native.EINVAL
    assert adj(A, 32, native.F32, 64, 32, 1e-6) == native.EINVAL         # lda < m
    assert adj(A, 64, native.F32, 64, 32, float("nan")) == native.EINVAL
    assert adj(A, 66, native.F32, 66, 32, 1e-6) == native.EINVAL         # lda * 4 not a multiple of 16
    assert adj(C.c_void_p(260), 64, native.F32, 64, 32, 1e-6) == native.EINVAL  # misaligned A
    assert b"aligned" in err()

    # no-allocation residual
    r = C.c_void_p(1024)
    assert L.asyflexa_residual_noalloc(None, x, r, None) == native.EINVAL
    q = native.Problem()
    q.m, q.n, q.lda = 64, 32, 64
    q.a_dtype, q.x_dtype = native.F32, native.F64
    q.A = q.b = 256
    assert L.asyflexa_residual_noalloc(C.byref(q), x, r, None) == native.EINVAL
    assert b"x_dtype" in err()
    q.x_dtype = native.F32
    q.a_dtype = native.BF16                # BF16 storage without column scales
    assert L.asyflexa_residual_noalloc(C.byref(q), x, r, None) == native.EINVAL
    assert b"col_scale" in err()
    q.a_dtype = native.F32
    q.n = 1 << 20                          # beyond the stated column limit
    assert L.asyflexa_residual_noalloc(C.byref(q), x, r, None) == native.EINVAL
    assert b"no-allocation limit" in err()
