"""Loader for the multi-core CPU oracle (``cores.c``): the partitioned lock-free form of
Algorithm 1 for LASSO (Section 4.2), FP64, timed against the number of cores, with the
threads sharing the residual r = Ax - b (residual form) or x with A^T A precomputed (Gram
form, the setup of the paper's experiments).

TEST INFRASTRUCTURE ONLY (see ``cores.c``).  The library is compiled with gcc
on first use into ``oracle/_build/``.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "cores.c")
LIB = os.path.join(_HERE, "_build", "liboracle_cores.so")
GCC_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off"]

_lib = None


def build() -> str:
    """Compile ``cores.c`` if the library is missing or older than the source."""
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *GCC_FLAGS, SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        f = lib.oracle_cores_lasso
        i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        f.argtypes = [i64, i64, i64, ptr, ptr, ptr, ptr, dbl, dbl, dbl, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      dbl, dbl, ptr, ptr]
        f.restype = ctypes.c_int
        _lib = lib
    return _lib


def gram(At, b, m: int, panel: int = 2048):
    """Q = A^T A (n x n) and q = A^T b in FP64 from the (n, lda) column store (numpy matmul,
    Q formed in row panels of ``panel`` rows on and right of the diagonal, then mirrored)."""
    A = np.asarray(At)[:, :m].astype(np.float64)
    n = A.shape[0]
    Q = np.empty((n, n))
    for j0 in range(0, n, panel):
        j1 = min(n, j0 + panel)
        Q[j0:j1, j0:] = A[j0:j1] @ A[j0:].T
        Q[j1:, j0:j1] = Q[j0:j1, j1:].T
    return Q, A @ np.asarray(b, dtype=np.float64)[:m]


def partitioned_lasso(At, b, m: int, lam: float, gamma: float = 0.9, tau: float = 0.0, w: int = 1,
                      threads: int = 1, max_sweeps: int = 100, f_star: float = math.nan, tol: float = 0.0,
                      x0=None, Q=None, q=None):
    """Partitioned asynchronous LASSO solve on ``threads`` host threads.

    ``At`` is the (n, lda) float32 column-major store (row j = column a_j, rows >= m unused),
    ``b`` the length-m data vector (converted to FP64).  ``Q``, ``q`` from :func:`gram` select
    the Gram form.  Stops when (F - f_star) / |f_star| < tol after a sweep (never for f_star
    NaN) or after ``max_sweeps`` sweeps.  Returns x (FP64) and a dict with sweeps, F (from
    r = Ax - b formed anew), F_running (F at the last check), seconds (wall time of the
    iteration without the checks), check_seconds and block_updates.
    """
    At = np.ascontiguousarray(At, dtype=np.float32)
    n, lda = At.shape
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64)[:m])
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    if (Q is None) != (q is None):
        raise ValueError("Q and q go together")
    qp = qq = None
    if Q is not None:
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        if Q.shape != (n, n) or q.shape != (n,):
            raise ValueError("Q must be n x n and q of length n")
        qp, qq = Q.ctypes.data, q.ctypes.data
    out = np.zeros(6)
    rc = _load().oracle_cores_lasso(m, n, lda, At.ctypes.data, b.ctypes.data, qp, qq, float(lam), float(gamma),
                                    float(tau), int(w), int(threads), int(max_sweeps), float(f_star), float(tol),
                                    x.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_cores_lasso rejected its arguments (rc {rc})")
    return x, {"sweeps": int(out[0]), "F": float(out[1]), "seconds": float(out[2]),
               "block_updates": int(out[3]), "F_running": float(out[4]), "check_seconds": float(out[5])}
