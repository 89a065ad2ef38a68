"""torch.autograd.Function for the LASSO solution map x*(lam, b) (argument marshalling only).

Forward: solve min 0.5||Ax - b||^2 + lam||x||_1 with the library (asyflexa_solve).
Backward, given v = dL/dx*: on the support S of x* with signs s the optimality conditions
A_S^T (A_S x_S - b) + lam s = 0 are smooth in (lam, b), so with w solving
(A_S^T A_S) w = v_S,
    dL/dlam = -s^T w,     dL/db = A_S w.
The library computes both in one call (asyflexa_adjoint): it selects S by
|x_j| > SUPPORT_REL_TOL * max(1, ||x||_inf), gathers A_S, runs its own block update on
    min_w 0.5||A_S w||^2 - v_S^T w      (b = 0, lam = 0, linear term -v_S),
whose minimiser solves the system above, and returns -s^T w and the exact residual A_S w.
Valid where the support and the signs of x* are locally constant.
"""

from __future__ import annotations

import ctypes as C

import torch

from . import native
from .native import AsyflexaError, Solver, lib

# The fixed step leaves geometric tails (1 - gamma)^k on coordinates that are zero at the
# optimum; the support excludes them with this relative threshold.
SUPPORT_REL_TOL = 1e-5

# The support problem is small: one CTA runs exact cyclic Gauss-Seidel on it.
ADJOINT_DEFAULTS = dict(mode="async", num_ctas=1, block_w=8, gamma=1.0, max_sweeps=2000, check_every=5,
                        refresh_every=5, tol_stat=1e-6)


def gather_columns(At, idx, m: int):
    """Columns idx of the column-major matrix At (n, lda) as a new (k, lda) tensor (library kernel)."""
    idx32 = idx.to(torch.int32).contiguous()
    k = int(idx32.numel())
    out = torch.empty((k, At.shape[1]), dtype=At.dtype, device=At.device)
    if k == 0:
        return out
    code = native._dtype_code(At)
    rc = lib().asyflexa_gather_columns(At.data_ptr(), At.shape[1], code, m, idx32.data_ptr(), k, out.data_ptr(),
                                       At.shape[1], C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != native.OK:
        raise AsyflexaError(rc, lib().asyflexa_last_error(None).decode())
    return out


def adjoint(At, m: int, x, v, rel_tol: float = SUPPORT_REL_TOL, **opts):
    """(dL/dlam, dL/db, |S|, stats of the support solve) for v = dL/dx* at the solution x
    (asyflexa_adjoint).  x and v: (n,) CUDA tensors of x's dtype; dL/db is FP64 (m,)."""
    if At.dim() != 2 or not At.is_contiguous():
        raise ValueError("At must be a contiguous (n, lda) CUDA tensor")
    xt = x.detach().contiguous()
    vt = v.detach().to(xt.dtype).contiguous()
    db = torch.empty(m, dtype=torch.float64, device=x.device)
    dlam = C.c_double(0.0)
    k = C.c_int64(0)
    st = native.Stats()
    o = native.make_opts(**dict(ADJOINT_DEFAULTS, **opts))
    rc = lib().asyflexa_adjoint(At.data_ptr(), At.shape[1], native._dtype_code(At), m, At.shape[0], xt.data_ptr(),
                                vt.data_ptr(), float(rel_tol), C.byref(o), C.byref(dlam), db.data_ptr(),
                                C.byref(k), C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc not in (native.OK, native.ENOTCONV):
        raise AsyflexaError(rc, lib().asyflexa_last_error(None).decode())
    return dlam.value, db, int(k.value), st.as_dict()


class LassoSolution(torch.autograd.Function):
    """x* = LassoSolution.apply(lam, b, At, m, solve_kwargs, adjoint_kwargs)."""

    @staticmethod
    def forward(ctx, lam, b, At, m, solve_kwargs, adjoint_kwargs):
        n = At.shape[0]
        s = Solver(At, b.detach().contiguous(), float(lam), m=m, **solve_kwargs)
        x = torch.zeros(n, dtype=torch.float32, device=At.device)
        st = s.solve(x)
        s.close()
        if st["status"] != native.OK:
            raise AsyflexaError(st["status"], f"forward solve did not converge: {st}")
        ctx.save_for_backward(x)
        ctx.At, ctx.m, ctx.adjoint_kwargs = At, m, adjoint_kwargs
        ctx.lam_like = lam
        ctx.b_dtype = b.dtype
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        dlam, db, _, _ = adjoint(ctx.At, ctx.m, x, gx, **(ctx.adjoint_kwargs or {}))
        lam_like = ctx.lam_like
        g_lam = torch.tensor(dlam, dtype=lam_like.dtype, device=x.device).reshape(lam_like.shape) \
            if torch.is_tensor(lam_like) else None
        return g_lam, db.to(ctx.b_dtype), None, None, None, None


def lasso_solution(lam, b, At, m: int, solve_kwargs: dict | None = None, adjoint_kwargs: dict | None = None):
    """Differentiable LASSO solution x*(lam, b) (lam: 0-d tensor, b: (m,) float32 tensor)."""
    return LassoSolution.apply(lam, b, At, m, solve_kwargs or {}, adjoint_kwargs or {})
