"""torch.autograd.Function around the solve, with the hand-written adjoint.

Forward: set the matrix values from the COO value vector v (Sec. 5 numeric
stage), solve A x = b with the fused PCG.  Backward: one adjoint solve
A^T lambda = dL/dx with the same kernels, then dL/db = lambda and
dL/dv_k = -lambda_{i_k} x_{j_k} for every kept COO entry (0 for ignored ones).
Gradients with respect to parameters that generate v (e.g. edge
conductivities) follow by ordinary autograd through the user's generator.

The matrix handle is shared state: forward leaves the values of v in it, and
backward assumes they are still there (do not set other values on the same
handle between forward and backward).  A must be symmetric.
"""
from __future__ import annotations

import torch

from . import binding as B


class SolveCG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, b, mat: B.Mat, opts: dict, batched: bool = False):
        mat.set_values(v.detach().contiguous())
        b = b.detach().contiguous()
        if batched:
            x, res = mat.solve_batched(b, **opts)
        else:
            x, r = mat.solve(b, **opts)
            res = [r]
        bad = [q for q in res if q["status"] != B.OK]
        if bad:
            raise B.GbsError(bad[0]["status"], "forward solve did not converge")
        ctx.mat, ctx.opts, ctx.batched = mat, opts, batched
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, _, dldv, res = ctx.mat.adjoint(x, gx.contiguous(), dlda=False, dldv=True,
                                            batched=ctx.batched, **ctx.opts)
        bad = [q for q in res if q["status"] != B.OK]
        if bad:
            raise B.GbsError(bad[0]["status"], "adjoint solve did not converge")
        return dldv, lam, None, None, None


def solve(v: torch.Tensor, b: torch.Tensor, mat: B.Mat, batched: bool = False, **opts):
    """x(v, b) = A(v)^{-1} b, differentiable in v and b."""
    return SolveCG.apply(v, b, mat, opts, batched)
