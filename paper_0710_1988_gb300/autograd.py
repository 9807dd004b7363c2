"""torch.autograd.Function for x = A^{-1} b (not in the paper: the
differentiation growth line).

Forward: D-BiCGStab (or plain BiCGStab) through the C ABI.  Backward, for an
incoming gradient g = dL/dx (PyTorch's convention dL = Re(g^dagger dx)):
lambda = A^{-dagger} g by one more solve through gamma5-hermiticity
(A^dagger = gamma5 A(-mu) gamma5, Sec. 1), then dL/db = lambda,
dL/dkappa = Re(lambda^dagger D x) and the link force dL/domega, all in the
library's kernels.  Only the solution x is kept between forward and
backward; no Krylov history is stored.
"""
from __future__ import annotations

import torch


class WilsonSolve(torch.autograd.Function):
    """x = WilsonSolve.apply(b, kappa, omega, op, deflation, tol, max_iter, mixed).

    b: complex128 CUDA tensor (12V elements).  kappa: 0-dim float64 tensor,
    equal to op.kappa.  omega: float64 tensor of shape (V, 4, 8), all zero: the
    Lie-algebra coordinates of the links around the operator's own links
    (U -> exp(i omega_a lambda_a / 2) U); its gradient is the link force.
    mixed: solve forward and adjoint with the mixed-precision solver (FP32 or
    FP16 iteration, FP64 true residual); the gradients are formed in FP64.
    """

    @staticmethod
    def forward(ctx, b, kappa, omega, op, deflation=None, tol=1e-10, max_iter=100000,
                mixed=False):
        if abs(float(kappa) - op.kappa) > 1e-15 * max(1.0, abs(op.kappa)):
            raise ValueError("kappa must equal the operator's kappa")
        if omega.abs().max().item() != 0.0:
            raise ValueError("omega must be zero: the gradient is taken at the operator's links")
        x = torch.zeros_like(b)
        solve = op.dbicgstab_mixed if mixed else op.dbicgstab
        rc, st = solve(b.contiguous(), x, deflation, tol=tol, max_iter=max_iter)
        if rc != 0:
            raise RuntimeError(f"forward solve failed (status {rc})")
        ctx.save_for_backward(x)
        ctx.op, ctx.deflation, ctx.tol, ctx.max_iter = op, deflation, tol, max_iter
        ctx.mixed = mixed
        ctx.omega_shape = omega.shape
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        op = ctx.op
        lam = torch.zeros_like(g)
        rc, st = op.adjoint_solve(g.contiguous(), lam, ctx.deflation, tol=ctx.tol,
                                  max_iter=ctx.max_iter, mixed=ctx.mixed)
        if rc != 0:
            raise RuntimeError(f"adjoint solve failed (status {rc})")
        want_k = ctx.needs_input_grad[1]
        want_w = ctx.needs_input_grad[2]
        force = (torch.empty(ctx.omega_shape, dtype=torch.float64, device=g.device)
                 if want_w else None)
        dk = op.gradients(lam, x, force=force, want_dkappa=want_k) if (want_k or want_w) else None
        grad_b = lam if ctx.needs_input_grad[0] else None
        grad_k = torch.tensor(dk, dtype=torch.float64) if want_k else None
        return grad_b, grad_k, force, None, None, None, None, None


def wilson_solve(b, kappa, omega, op, deflation=None, tol=1e-10, max_iter=100000, mixed=False):
    return WilsonSolve.apply(b, kappa, omega, op, deflation, tol, max_iter, mixed)
