"""torch.autograd.Function for the LASSO solution map x*(lam, b) (argument marshalling only).

Forward: solve min 0.5||Ax - b||^2 + lam||x||_1 with the library (asyflexa_solve).
Backward, given v = dL/dx*: on the support S of x* with signs s the optimality conditions
A_S^T (A_S x_S - b) + lam s = 0 are smooth in (lam, b), so with w solving
(A_S^T A_S) w = v_S,
    dL/dlam = -s^T w,     dL/db = A_S w.
w is computed by the library's own block update restricted to the support: the columns A_S
are gathered (asyflexa_gather_columns) and the method is run on
    min_w 0.5||A_S w||^2 - v_S^T w      (b = 0, lam = 0, linear term -v_S),
whose minimiser solves the system above; the exact residual of that run is A_S w = dL/db.
Valid where the support and the signs of x* are locally constant.
"""

from __future__ import annotations

import ctypes as C

import torch

from . import native
from .native import AsyflexaError, Solver, lib

SUPPORT_REL_TOL = 1e-5


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


def support(x, rel_tol: float = SUPPORT_REL_TOL):
    """Indices with |x_j| > rel_tol * max(1, ||x||_inf) (the fixed step leaves geometric
    tails (1 - gamma)^k on coordinates that are zero at the optimum; they are excluded)."""
    scale = max(1.0, float(x.abs().max())) if x.numel() else 1.0
    return torch.nonzero(x.abs() > rel_tol * scale).flatten()


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
        At, m = ctx.At, ctx.m
        S = support(x)
        k = int(S.numel())
        dlam = torch.zeros((), dtype=torch.float64, device=x.device)
        db = torch.zeros(m, dtype=torch.float64, device=x.device)
        if k > 0:
            AS = gather_columns(At, S, m)
            lin = (-gx[S]).to(torch.float32).contiguous()
            zero_b = torch.zeros(m, dtype=torch.float32, device=x.device)
            kw = dict(mode="async", num_ctas=1, block_w=8, gamma=1.0, max_sweeps=2000, check_every=5,
                      refresh_every=5, tol_stat=1e-6)
            kw.update(ctx.adjoint_kwargs or {})
            adj = Solver(AS, zero_b, 0.0, m=m, lin=lin, **kw)
            w = torch.zeros(k, dtype=torch.float32, device=x.device)
            st = adj.solve(w)
            if st["status"] not in (native.OK, native.ENOTCONV):
                raise AsyflexaError(st["status"], "adjoint solve failed")
            db = adj.residual()                      # A_S w - 0, FP64
            adj.close()
            dlam = -(torch.sign(x[S]).double() * w.double()).sum()
        lam_like = ctx.lam_like
        g_lam = dlam.to(lam_like.dtype).reshape(lam_like.shape) if torch.is_tensor(lam_like) else None
        return g_lam, db.to(ctx.b_dtype), None, None, None, None


def lasso_solution(lam, b, At, m: int, solve_kwargs: dict | None = None, adjoint_kwargs: dict | None = None):
    """Differentiable LASSO solution x*(lam, b) (lam: 0-d tensor, b: (m,) float32 tensor)."""
    return LassoSolution.apply(lam, b, At, m, solve_kwargs or {}, adjoint_kwargs or {})
