"""ctypes wrapper of the batched C ABI (asyflexa_batch_*), argument marshalling only."""

from __future__ import annotations

import ctypes as C
import math

from . import native
from .native import AsyflexaError, Problem, Stats, default_opts, lib


FORMS = {"auto": 0, "async": native.BATCH_FORM_ASYNC, "gs": native.BATCH_FORM_GS, "multi": native.BATCH_FORM_MULTI}


class BatchSolver:
    """Many FP32 problems solved together (asyflexa_batch_*).

    ``problems``: list of dicts with keys At (n, lda) CUDA float32, b, lam, m and optional
    lo, hi, lin, loss ("lasso"/"ncquad"), c.  ``form``: "gs" (one persistent launch, one CTA
    per problem at a time, exact Gauss-Seidel with in-kernel stopping tests), "async" (rounds
    of the asynchronous kernel over all problems' blocks) or "auto".  ``block_w = 0``
    autotunes the block width of the async rounds.  ``shared_a``: the problems share one
    matrix.
    """

    def __init__(self, problems, *, block_w=32, gamma=0.9, tau=0.0, tau_rel=0.0, refresh_every=10,
                 check_every=10, max_sweeps=1000, num_ctas=0, tol_gap=1e-6, tol_stat=1e-6, switch_tol=1e-9,
                 shared_a=False, form="auto", stream=None):
        import torch
        L = lib()
        n = len(problems)
        arr = (Problem * n)()
        self._keep = []
        for k, pr in enumerate(problems):
            At = pr["At"]
            p = arr[k]
            p.m, p.n, p.lda = int(pr["m"]), At.shape[0], At.shape[1]
            p.a_dtype = p.x_dtype = native.F32
            p.A, p.b = At.data_ptr(), pr["b"].data_ptr()
            for key in ("lo", "hi", "lin"):
                if pr.get(key) is not None:
                    setattr(p, key, pr[key].data_ptr())
            p.lam, p.c = float(pr["lam"]), float(pr.get("c", 0.0))
            p.loss = native.LOSSES[pr.get("loss", "lasso")]
            self._keep.append(pr)
        o = default_opts()
        o.block_w, o.mode, o.gamma, o.tau, o.tau_rel = int(block_w), native.ASYNC, float(gamma), float(tau), float(tau_rel)
        o.refresh_every, o.max_sweeps, o.num_ctas = int(refresh_every), int(max_sweeps), int(num_ctas)
        o.check_every = int(check_every)
        o.tol_gap, o.tol_stat, o.switch_tol = float(tol_gap), float(tol_stat), float(switch_tol)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        if form not in FORMS:
            raise ValueError(f"form must be one of {sorted(FORMS)}")
        flags = (native.BATCH_SHARED_A if shared_a else 0) | FORMS[form]
        h = C.c_void_p()
        rc = L.asyflexa_batch_create(C.byref(h), arr, n, C.byref(o), flags, C.c_void_p(stream))
        if rc != native.OK:
            raise AsyflexaError(rc, L.asyflexa_last_error(None).decode())
        self.h, self.count, self.problems = h, n, arr

    def solve(self, xs, f_star=None):
        """Solve in place; returns (per-problem stats list, total stats dict)."""
        L = lib()
        ptrs = (C.c_void_p * self.count)(*[x.data_ptr() for x in xs])
        fs = None
        if f_star is not None:
            fs = (C.c_double * self.count)(*[math.nan if v is None else float(v) for v in f_star])
        per = (Stats * self.count)()
        tot = Stats()
        rc = L.asyflexa_batch_solve(self.h, ptrs, fs, per, C.byref(tot))
        # ENOTCONV / ENONFINITE describe problems (their own status is in per): not raised
        if rc < 0 and rc != native.ENONFINITE:
            raise AsyflexaError(rc, L.asyflexa_last_error(None).decode())
        return [s.as_dict() for s in per], tot.as_dict()

    def check(self, xs, f_star=None):
        """The library's exact check (asyflexa_check) of every problem at xs; list of dicts."""
        L = lib()
        ptrs = (C.c_void_p * self.count)(*[x.data_ptr() for x in xs])
        fs = None
        if f_star is not None:
            fs = (C.c_double * self.count)(*[math.nan if v is None else float(v) for v in f_star])
        per = (Stats * self.count)()
        rc = L.asyflexa_batch_check(self.h, ptrs, fs, per)
        if rc != native.OK:
            raise AsyflexaError(rc, L.asyflexa_last_error(None).decode())
        return [s.as_dict() for s in per]

    def close(self):
        if getattr(self, "h", None):
            lib().asyflexa_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiLaneSolver:
    """k LASSO lanes sharing one FP32 matrix (a lambda path or several data vectors), every
    block update done for all lanes at once on the tensor cores (asyflexa_multi_*).

    ``At`` (n, lda) CUDA float32; ``B`` (k, m) CUDA float32 (row l = lane l's b); ``lambdas``
    k floats.  ``solve(X)`` takes X (k, n) CUDA float32 (row l = lane l's x), in place.
    """

    def __init__(self, At, B, lambdas, m, *, gamma=0.9, tau=0.0, tau_rel=0.0, refresh_every=10, check_every=10,
                 max_sweeps=1000, num_ctas=0, tol_gap=1e-6, tol_stat=1e-6, switch_tol=1e-9, stream=None):
        import torch
        L = lib()
        if At.dtype != torch.float32 or not At.is_contiguous() or not At.is_cuda:
            raise ValueError("At must be a contiguous float32 CUDA tensor (n, lda)")
        if B.dtype != torch.float32 or not B.is_contiguous() or B.dim() != 2:
            raise ValueError("B must be a contiguous float32 CUDA tensor (k, ldb)")
        n, lda = At.shape
        k = B.shape[0]
        p = Problem()
        p.m, p.n, p.lda = int(m), n, lda
        p.a_dtype = p.x_dtype = native.F32
        p.A, p.b = At.data_ptr(), B.data_ptr()
        p.loss = native.LOSS_LASSO
        o = default_opts()
        o.mode, o.gamma, o.tau, o.tau_rel = native.ASYNC, float(gamma), float(tau), float(tau_rel)
        o.refresh_every, o.check_every, o.max_sweeps, o.num_ctas = int(refresh_every), int(check_every), \
            int(max_sweeps), int(num_ctas)
        o.tol_gap, o.tol_stat, o.switch_tol = float(tol_gap), float(tol_stat), float(switch_tol)
        lam = (C.c_double * k)(*[float(v) for v in lambdas])
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        rc = L.asyflexa_multi_create(C.byref(h), C.byref(p), k, B.data_ptr(), B.shape[1], lam, C.byref(o),
                                     C.c_void_p(stream))
        if rc != native.OK:
            raise AsyflexaError(rc, L.asyflexa_last_error(None).decode())
        self.h, self.k, self.n = h, k, n
        self._keep = (At, B)

    def solve(self, X, f_star=None):
        """Solve every lane from X (k, ldx) in place; returns (per-lane stats, total stats)."""
        L = lib()
        if X.shape[0] != self.k or X.shape[1] < self.n or not X.is_contiguous():
            raise ValueError("X must be a contiguous (k, >= n) float32 CUDA tensor")
        fs = None
        if f_star is not None:
            fs = (C.c_double * self.k)(*[math.nan if v is None else float(v) for v in f_star])
        per = (Stats * self.k)()
        tot = Stats()
        rc = L.asyflexa_multi_solve(self.h, X.data_ptr(), X.shape[1], fs, per, C.byref(tot))
        if rc < 0:
            raise AsyflexaError(rc, L.asyflexa_last_error(None).decode())
        return [s.as_dict() for s in per], tot.as_dict()

    def close(self):
        if getattr(self, "h", None):
            lib().asyflexa_multi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
