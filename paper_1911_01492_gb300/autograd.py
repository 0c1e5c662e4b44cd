"""Differentiable operator application and solve (torch.autograd.Function).

Both functions take log K (the coefficient at the volume Gauss points, CUDA
float64) as an input so that gradients flow to it.  The mesh's coefficient is
derived from it (dg_set_coefficient) only when it differs from the log K the
mesh was last set from by these functions: each call compares log K exactly
with a private copy of that last value (one device comparison), so repeated
applies and solves with an unchanged coefficient skip the setup.

apply(x, logK, mesh) = A(K) x
    d/dx:     A^T ybar                      (dg_apply_adjoint)
    d/dlogK:  d(ybar^T A x)/dlogK           (dg_coeff_grad(u = x, v = ybar))
solve(b, logK, mesh) = A(K)^{-1} b   by CG
    d/db:     lambda = A^{-T} ubar          (one adjoint CG solve; A is symmetric)
    d/dlogK:  -d(lambda^T A u)/dlogK        (dg_coeff_grad(u, lambda))
No iterate of the forward solve is stored: the backward pass is a fresh solve.
"""
from __future__ import annotations

import torch

from . import DG_CG_FP64, DG_CG_PRECOND_JACOBI, Mesh


def _ensure_coefficient(mesh: Mesh, logK: torch.Tensor):
    # An exact comparison with a private copy, not the version counter: a
    # tensor's values can change without its version (writes through .data).
    # Mesh.set_coefficient drops the copy, so a coefficient set directly by the
    # caller is never mistaken for this one.
    lk = logK.detach()
    last = mesh._autograd_logK
    if (last is not None and last.shape == lk.shape and last.device == lk.device
            and torch.equal(last, lk)):
        return
    mesh.set_coefficient(torch.exp(lk).contiguous())
    mesh._autograd_logK = lk.clone()


class ApplyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, logK, mesh):
        _ensure_coefficient(mesh, logK)
        ctx.mesh = mesh
        ctx.save_for_backward(x, logK)
        return mesh.apply(x.detach().contiguous())

    @staticmethod
    def backward(ctx, ybar):
        x, logK = ctx.saved_tensors
        mesh = ctx.mesh
        _ensure_coefficient(mesh, logK)
        ybar = ybar.contiguous()
        gx = mesh.apply_adjoint(ybar) if ctx.needs_input_grad[0] else None
        gk = None
        if ctx.needs_input_grad[1]:
            gk = mesh.coeff_grad(x.detach().double().contiguous(), ybar.double().contiguous())
        return gx, gk, None


class SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, logK, mesh, rtol, mode):
        _ensure_coefficient(mesh, logK)
        u, st = mesh.cg_solve(b.detach().contiguous(), rtol=rtol, mode=mode)
        ctx.mesh, ctx.rtol, ctx.mode = mesh, rtol, mode
        ctx.stats = st
        ctx.save_for_backward(u, logK)
        return u

    @staticmethod
    def backward(ctx, ubar):
        u, logK = ctx.saved_tensors
        mesh = ctx.mesh
        _ensure_coefficient(mesh, logK)
        lam, st = mesh.cg_solve(ubar.contiguous(), rtol=ctx.rtol, mode=ctx.mode)
        gb = lam if ctx.needs_input_grad[0] else None
        gk = -mesh.coeff_grad(u, lam) if ctx.needs_input_grad[1] else None
        return gb, gk, None, None, None


def apply(x: torch.Tensor, logK: torch.Tensor, mesh: Mesh) -> torch.Tensor:
    """y = A(exp(logK)) x, differentiable in x (float64 or float32) and logK."""
    return ApplyFn.apply(x, logK, mesh)


def solve(b: torch.Tensor, logK: torch.Tensor, mesh: Mesh, rtol: float = 1e-12,
          mode: int = DG_CG_FP64, precond: str | None = None) -> torch.Tensor:
    """u = A(exp(logK))^{-1} b by CG, differentiable in b and logK (adjoint CG).
    mode and precond (None or "jacobi") select the solver of both the forward
    and the adjoint solve, as in Mesh.cg_solve."""
    if precond not in (None, "jacobi"):
        raise ValueError(f"unknown preconditioner {precond!r}")
    if precond == "jacobi":
        mode |= DG_CG_PRECOND_JACOBI
    return SolveFn.apply(b, logK, mesh, rtol, mode)
