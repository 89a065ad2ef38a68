"""ctypes binding of the C ABI in ``include/asyflexa.h`` (argument marshalling only).

The functions keep the C names (``asyflexa_create``, ``asyflexa_solve`` ...) on the
loaded library object returned by :func:`lib`.  :class:`Solver` is a thin convenience
wrapper that takes torch tensors for device memory and the current torch CUDA stream;
every step of the method runs in the library's CUDA kernels.  There is no fallback: if
the library is missing or cannot be loaded, importing or calling raises.
"""

from __future__ import annotations

import ctypes as C
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libasyflexa.so")

OK, ENOTCONV, EINVAL, ECUDA, ENOMEM, ETIMEOUT, ENONFINITE, EUNSUPPORTED = 0, 1, -1, -2, -3, -4, -5, -6
LOSS_LASSO, LOSS_NCQUAD, LOSS_DC_LOG, LOSS_DC_EXP = 0, 1, 2, 3
LOSSES = {"lasso": LOSS_LASSO, "ncquad": LOSS_NCQUAD, "dc_log": LOSS_DC_LOG, "dc_exp": LOSS_DC_EXP}
SYNC, ASYNC = 0, 1
F64, F32, BF16, FP8E4M3 = 0, 1, 2, 3


class Problem(C.Structure):
    _fields_ = [
        ("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64),
        ("a_dtype", C.c_int32), ("x_dtype", C.c_int32),
        ("A", C.c_void_p), ("col_scale", C.c_void_p), ("b", C.c_void_p),
        ("lo", C.c_void_p), ("hi", C.c_void_p),
        ("lam", C.c_double), ("c", C.c_double),
        ("loss", C.c_int32), ("reserved0", C.c_int32),
        ("A_master", C.c_void_p), ("lda_master", C.c_int64),
        ("lin", C.c_void_p),
    ]


class Opts(C.Structure):
    _fields_ = [
        ("block_w", C.c_int32), ("mode", C.c_int32),
        ("gamma", C.c_double), ("tau", C.c_double), ("tau_rel", C.c_double),
        ("refresh_every", C.c_int32), ("check_every", C.c_int32), ("max_sweeps", C.c_int32),
        ("num_ctas", C.c_int32),
        ("tol_gap", C.c_double), ("tol_stat", C.c_double), ("f_star", C.c_double),
        ("seed", C.c_uint64), ("profile", C.c_int32), ("variant", C.c_int32),
        ("switch_tol", C.c_double), ("gamma_mu", C.c_double),
        ("tau_adapt", C.c_int32), ("exact_grad", C.c_int32),
        ("delay_ns", C.c_int32), ("reserved2", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int64), ("block_updates", C.c_int64),
        ("F", C.c_double), ("rel_gap", C.c_double), ("stat_xhat", C.c_double), ("stat_mf", C.c_double),
        ("kkt_viol", C.c_double), ("nnz", C.c_int64), ("seconds", C.c_double), ("hbm_bytes", C.c_double),
        ("staleness_hist", C.c_uint64 * 32), ("kernel_launches", C.c_int64),
        ("sweep_kernel_seconds", C.c_double), ("sweep_kernel_launches", C.c_int64),
        ("sweep_kernel_sweeps", C.c_int64),
        ("status", C.c_int32), ("checked", C.c_int32),
        ("polish_sweeps", C.c_int64), ("polish_seconds", C.c_double),
        ("block_w", C.c_int32), ("kernel_variant", C.c_int32), ("dual_gap", C.c_double),
        ("tau_extra", C.c_double), ("batch_form", C.c_int32), ("ctas_per_sm", C.c_int32),
        ("handed_over", C.c_int32), ("reserved1", C.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["staleness_hist"] = list(self.staleness_hist)
        return d


_lib = None
EXPORTS = [
    "asyflexa_version", "asyflexa_status_string", "asyflexa_opts_default", "asyflexa_create",
    "asyflexa_destroy", "asyflexa_residual_refresh", "asyflexa_step", "asyflexa_solve", "asyflexa_check",
    "asyflexa_read_counters", "asyflexa_reset_counters", "asyflexa_get_residual", "asyflexa_get_weights",
    "asyflexa_last_error", "asyflexa_residual_noalloc", "asyflexa_quantize", "asyflexa_gather_columns",
    "asyflexa_batch_create", "asyflexa_batch_solve", "asyflexa_batch_check", "asyflexa_batch_destroy",
    "asyflexa_multi_create", "asyflexa_multi_solve", "asyflexa_multi_destroy",
    "asyflexa_convert_check", "asyflexa_wait_check", "asyflexa_adjoint",
]
BATCH_SHARED_A = 1
BATCH_FORM_ASYNC = 2
BATCH_FORM_GS = 4
BATCH_FORM_MULTI = 8


def lib(path: str | None = None):
    """Load ``libasyflexa.so`` (built in-tree by ``paper_1701_04900_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libasyflexa.so not found at {p}; build it with "
                          "`python -m paper_1701_04900_gb300.build` (no CPU fallback exists)")
    L = C.CDLL(p)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    L.asyflexa_version.restype = C.c_int
    L.asyflexa_status_string.restype = C.c_char_p
    L.asyflexa_status_string.argtypes = [C.c_int]
    L.asyflexa_opts_default.restype = None
    L.asyflexa_opts_default.argtypes = [C.POINTER(Opts)]
    L.asyflexa_create.restype = C.c_int
    L.asyflexa_create.argtypes = [C.POINTER(vp), C.POINTER(Problem), C.POINTER(Opts), vp]
    L.asyflexa_destroy.restype = C.c_int
    L.asyflexa_destroy.argtypes = [vp]
    L.asyflexa_residual_refresh.restype = C.c_int
    L.asyflexa_residual_refresh.argtypes = [vp, vp]
    L.asyflexa_step.restype = C.c_int
    L.asyflexa_step.argtypes = [vp, vp, i32]
    L.asyflexa_solve.restype = C.c_int
    L.asyflexa_solve.argtypes = [vp, vp, C.POINTER(Stats)]
    L.asyflexa_check.restype = C.c_int
    L.asyflexa_check.argtypes = [vp, vp, C.POINTER(Stats)]
    L.asyflexa_read_counters.restype = C.c_int
    L.asyflexa_read_counters.argtypes = [vp, C.POINTER(Stats)]
    L.asyflexa_reset_counters.restype = C.c_int
    L.asyflexa_reset_counters.argtypes = [vp]
    L.asyflexa_get_residual.restype = C.c_int
    L.asyflexa_get_residual.argtypes = [vp, vp]
    L.asyflexa_get_weights.restype = C.c_int
    L.asyflexa_get_weights.argtypes = [vp, vp]
    L.asyflexa_last_error.restype = C.c_char_p
    L.asyflexa_last_error.argtypes = [vp]
    L.asyflexa_residual_noalloc.restype = C.c_int
    L.asyflexa_residual_noalloc.argtypes = [C.POINTER(Problem), vp, vp, vp]
    L.asyflexa_convert_check.restype = C.c_int
    L.asyflexa_convert_check.argtypes = [i32, vp, vp, C.c_int64, vp]
    L.asyflexa_wait_check.restype = C.c_int
    L.asyflexa_wait_check.argtypes = [i32, C.c_int64, C.POINTER(C.c_int)]
    L.asyflexa_quantize.restype = C.c_int
    L.asyflexa_quantize.argtypes = [vp, C.c_int64, C.c_int64, C.c_int64, i32, vp, C.c_int64, vp, vp]
    L.asyflexa_batch_create.restype = C.c_int
    L.asyflexa_batch_create.argtypes = [C.POINTER(vp), C.POINTER(Problem), i32, C.POINTER(Opts), i32, vp]
    L.asyflexa_batch_solve.restype = C.c_int
    L.asyflexa_batch_solve.argtypes = [vp, C.POINTER(vp), vp, C.POINTER(Stats), C.POINTER(Stats)]
    L.asyflexa_batch_check.restype = C.c_int
    L.asyflexa_batch_check.argtypes = [vp, C.POINTER(vp), vp, C.POINTER(Stats)]
    L.asyflexa_batch_destroy.restype = C.c_int
    L.asyflexa_batch_destroy.argtypes = [vp]
    L.asyflexa_multi_create.restype = C.c_int
    L.asyflexa_multi_create.argtypes = [C.POINTER(vp), C.POINTER(Problem), i32, vp, C.c_int64, vp, C.POINTER(Opts), vp]
    L.asyflexa_multi_solve.restype = C.c_int
    L.asyflexa_multi_solve.argtypes = [vp, vp, C.c_int64, vp, C.POINTER(Stats), C.POINTER(Stats)]
    L.asyflexa_multi_destroy.restype = C.c_int
    L.asyflexa_multi_destroy.argtypes = [vp]
    L.asyflexa_gather_columns.restype = C.c_int
    L.asyflexa_gather_columns.argtypes = [vp, C.c_int64, i32, C.c_int64, vp, C.c_int64, vp, C.c_int64, vp]
    L.asyflexa_adjoint.restype = C.c_int
    L.asyflexa_adjoint.argtypes = [vp, C.c_int64, i32, C.c_int64, C.c_int64, vp, vp, dbl, C.POINTER(Opts),
                                   C.POINTER(dbl), vp, C.POINTER(C.c_int64), C.POINTER(Stats), vp]
    del dbl
    if path is None:
        _lib = L
    return L


class AsyflexaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{code} ({_status_name(code)}): {msg}")
        self.code = code


def _status_name(code: int) -> str:
    try:
        return lib().asyflexa_status_string(code).decode()
    except Exception:  # pragma: no cover
        return str(code)


def _dtype_code(t) -> int:
    import torch
    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16,
            torch.float8_e4m3fn: FP8E4M3}[t.dtype]


def default_opts() -> Opts:
    o = Opts()
    lib().asyflexa_opts_default(C.byref(o))
    return o


def make_opts(block_w=32, mode="sync", gamma=0.9, tau=0.0, tau_rel=0.0, refresh_every=10, check_every=10,
              max_sweeps=1000, num_ctas=0, tol_gap=1e-6, tol_stat=1e-6, f_star=math.nan, profile=False, variant=0,
              switch_tol=1e-7, gamma_mu=0.0, tau_adapt=False, exact_grad=0, delay_ns=0) -> Opts:
    """asyflexa_opts from keyword arguments (the library's defaults, then these values)."""
    o = default_opts()
    o.block_w, o.mode = int(block_w), (ASYNC if mode == "async" else SYNC)
    o.gamma, o.tau, o.tau_rel = float(gamma), float(tau), float(tau_rel)
    o.refresh_every, o.check_every, o.max_sweeps = int(refresh_every), int(check_every), int(max_sweeps)
    o.num_ctas = int(num_ctas)
    o.tol_gap, o.tol_stat, o.f_star = float(tol_gap), float(tol_stat), float(f_star)
    o.profile = 1 if profile else 0
    o.variant = int(variant)
    o.switch_tol = float(switch_tol)
    o.gamma_mu = float(gamma_mu)
    o.tau_adapt = 1 if tau_adapt else 0
    o.exact_grad = int(exact_grad)
    o.delay_ns = int(delay_ns)
    return o


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Solver:
    """One problem instance on the current CUDA device (a handle of the C ABI).

    ``At`` is the column-major matrix as a contiguous CUDA tensor of shape (n, lda):
    row j holds column a_j (only the first ``m`` entries are used).  ``b`` (m,), ``lo``,
    ``hi`` (n,) and the ``x`` passed to the methods are CUDA tensors of float64 (for
    float64 A) or float32 (otherwise).  The tensors must stay alive and unchanged while the
    solver exists (the wrapper keeps references).
    """

    def __init__(self, At, b, lam, m=None, *, loss="lasso", c=0.0, theta=None, lo=None, hi=None, col_scale=None,
                 block_w=32, mode="sync", gamma=0.9, tau=0.0, tau_rel=0.0, refresh_every=10,
                 check_every=10, max_sweeps=1000, num_ctas=0, tol_gap=1e-6, tol_stat=1e-6,
                 f_star=math.nan, profile=False, variant=0, A_master=None, switch_tol=1e-7, lin=None,
                 gamma_mu=0.0, tau_adapt=False, exact_grad=0, delay_ns=0, stream=None):
        import torch
        L = lib()
        if At.dim() != 2 or not At.is_contiguous() or not At.is_cuda:
            raise ValueError("At must be a contiguous (n, lda) CUDA tensor")
        n, lda = At.shape
        m = lda if m is None else int(m)
        self._keep = [At, b, lo, hi, col_scale, A_master, lin]
        p = Problem()
        p.m, p.n, p.lda = m, n, lda
        p.a_dtype = _dtype_code(At)
        p.x_dtype = F64 if p.a_dtype == F64 else F32
        p.A, p.col_scale, p.b = At.data_ptr(), (col_scale.data_ptr() if col_scale is not None else None), b.data_ptr()
        p.lo = lo.data_ptr() if lo is not None else None
        p.hi = hi.data_ptr() if hi is not None else None
        if loss not in LOSSES:
            raise ValueError(f"loss must be one of {sorted(LOSSES)}")
        p.loss = LOSSES[loss]
        # the DC losses take their regulariser parameter theta in the c field of the ABI
        p.lam, p.c = float(lam), float(theta if theta is not None else c)
        if lin is not None:
            p.lin = lin.data_ptr()
        if A_master is not None:
            if A_master.dtype != torch.float32 or not A_master.is_contiguous() or A_master.shape[0] != n:
                raise ValueError("A_master must be a contiguous float32 (n, lda_master) CUDA tensor")
            p.A_master, p.lda_master = A_master.data_ptr(), A_master.shape[1]
        o = make_opts(block_w=block_w, mode=mode, gamma=gamma, tau=tau, tau_rel=tau_rel, refresh_every=refresh_every,
                      check_every=check_every, max_sweeps=max_sweeps, num_ctas=num_ctas, tol_gap=tol_gap,
                      tol_stat=tol_stat, f_star=f_star, profile=profile, variant=variant, switch_tol=switch_tol,
                      gamma_mu=gamma_mu, tau_adapt=tau_adapt, exact_grad=exact_grad, delay_ns=delay_ns)
        self.problem, self.opts = p, o
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = C.c_void_p()
        rc = L.asyflexa_create(C.byref(h), C.byref(p), C.byref(o), C.c_void_p(stream))
        if rc != OK:
            raise AsyflexaError(rc, L.asyflexa_last_error(None).decode())
        self.h = h
        self.m, self.n = m, n

    # -- helpers
    def _err(self, rc):
        raise AsyflexaError(rc, lib().asyflexa_last_error(self.h).decode())

    def _check_x(self, x):
        import torch
        want = torch.float64 if self.problem.x_dtype == F64 else torch.float32
        if x.dtype != want or not x.is_cuda or not x.is_contiguous() or x.numel() != self.n:
            raise ValueError(f"x must be a contiguous CUDA {want} tensor of length {self.n}")

    # -- C-ABI calls
    def refresh(self, x):
        self._check_x(x)
        rc = lib().asyflexa_residual_refresh(self.h, x.data_ptr())
        if rc != OK:
            self._err(rc)

    def step(self, x, n_sweeps: int):
        self._check_x(x)
        rc = lib().asyflexa_step(self.h, x.data_ptr(), int(n_sweeps))
        if rc != OK:
            self._err(rc)

    def solve(self, x) -> dict:
        self._check_x(x)
        st = Stats()
        rc = lib().asyflexa_solve(self.h, x.data_ptr(), C.byref(st))
        if rc not in (OK, ENOTCONV):
            self._err(rc)
        return st.as_dict()

    def check(self, x) -> dict:
        self._check_x(x)
        st = Stats()
        rc = lib().asyflexa_check(self.h, x.data_ptr(), C.byref(st))
        if rc != OK:
            self._err(rc)
        return st.as_dict()

    def read_counters(self) -> dict:
        st = Stats()
        rc = lib().asyflexa_read_counters(self.h, C.byref(st))
        if rc != OK:
            self._err(rc)
        return st.as_dict()

    def reset_counters(self):
        rc = lib().asyflexa_reset_counters(self.h)
        if rc != OK:
            self._err(rc)

    def residual(self):
        import torch
        out = torch.empty(self.m, dtype=torch.float64, device="cuda")
        rc = lib().asyflexa_get_residual(self.h, out.data_ptr())
        if rc != OK:
            self._err(rc)
        return out

    def weights(self):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        rc = lib().asyflexa_get_weights(self.h, out.data_ptr())
        if rc != OK:
            self._err(rc)
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().asyflexa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def convert_check(src, stream=None, storage: str | None = None):
    """The kernels' own conversions (asyflexa_convert_check) applied to a CUDA tensor:
    float64 -> float32 (round to nearest even), float32 -> float64 (exact), or, with
    ``storage`` = "fp8" / "bf16", the decoding of stored A elements (a uint8 tensor of e4m3
    codes or a bfloat16 tensor) to float32."""
    import torch
    if not src.is_cuda or not src.is_contiguous():
        raise ValueError("src must be a contiguous CUDA tensor")
    if storage is None:
        if src.dtype not in (torch.float64, torch.float32):
            raise ValueError("src must be float64 or float32")
        d = 0 if src.dtype == torch.float64 else 1
        out = torch.empty(src.shape, dtype=torch.float32 if d == 0 else torch.float64, device=src.device)
    elif storage in ("fp8", "bf16"):
        want = torch.uint8 if storage == "fp8" else torch.bfloat16
        if src.dtype != want:
            raise ValueError(f"storage {storage!r} takes a {want} tensor")
        d = 2 if storage == "fp8" else 3
        out = torch.empty(src.shape, dtype=torch.float32, device=src.device)
    else:
        raise ValueError("storage must be None, 'fp8' or 'bf16'")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    rc = lib().asyflexa_convert_check(d, src.data_ptr(), out.data_ptr(), src.numel(), C.c_void_p(stream))
    if rc != OK:
        raise AsyflexaError(rc, lib().asyflexa_last_error(None).decode())
    return out


def wait_check(arrive_first: bool, limit_ns: int):
    """The kernels' bounded mbarrier wait in a one-thread kernel (asyflexa_wait_check):
    returns (status, completed, recorded error, abort flag, elapsed microseconds)."""
    res = (C.c_int * 4)()
    rc = lib().asyflexa_wait_check(1 if arrive_first else 0, int(limit_ns), res)
    if rc not in (OK, ETIMEOUT):
        raise AsyflexaError(rc, lib().asyflexa_last_error(None).decode())
    return rc, res[0], res[1], res[2], res[3]


def quantize(At, m: int, kind: str, stream=None):
    """Per-column scaled BF16 / FP8-e4m3 copy of a float32 (n, lda) CUDA matrix by the
    library's kernel (asyflexa_quantize).  Returns (Q of shape (n, ldq), scale (n,))."""
    import torch
    if At.dtype != torch.float32 or not At.is_cuda or not At.is_contiguous():
        raise ValueError("At must be a contiguous float32 CUDA tensor")
    n, lda = At.shape
    if kind == "bf16":
        tdt, code, per = torch.bfloat16, BF16, 8
    elif kind == "fp8":
        tdt, code, per = torch.float8_e4m3fn, FP8E4M3, 16
    else:
        raise ValueError(kind)
    ldq = (m + per - 1) // per * per
    Q = torch.empty((n, ldq), dtype=tdt, device=At.device)
    scale = torch.empty(n, dtype=torch.float32, device=At.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    rc = lib().asyflexa_quantize(At.data_ptr(), m, n, lda, code, Q.data_ptr(), ldq, scale.data_ptr(),
                                 C.c_void_p(stream))
    if rc != OK:
        raise AsyflexaError(rc, lib().asyflexa_last_error(None).decode())
    return Q, scale
