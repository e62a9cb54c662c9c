"""Differentiable kernel ridge regression on the Nystrom PCG library.

The training system (K + mu I) alpha = b (Sec. 6.5, Eq. (6.3), with mu the
diagonal actually added) is solved by Nystrom PCG; its gradient comes from one
more solve with the same matrix (the adjoint), preconditioned by the same
Nystrom factor:

    lambda     = (K + mu I)^{-1} g            g = dL/dalpha
    dL/db      = lambda
    dL/dmu     = -lambda^T alpha
    dL/dsigma  = -lambda^T (dK/dsigma) alpha,   dK_ij/dsigma = K_ij ||x_i-x_j||^2 / sigma^3

Predictions K_v alpha on validation points have the adjoint K_v^T g and the
sigma-derivative g^T (dK_v/dsigma) alpha.  Every product runs in the CUDA
library; this module only wires them into torch.autograd.
"""

from __future__ import annotations

import torch

from . import nyspcg as ny


def _scalar(x) -> float:
    return float(x.detach().item()) if torch.is_tensor(x) else float(x)


class KRRSolve(torch.autograd.Function):
    """alpha = (K_sigma + mu I)^{-1} b with a Nystrom-preconditioned solve."""

    @staticmethod
    def forward(ctx, b, mu, sigma, points, ell, precision, tol, seed):
        mu_f, sig_f = _scalar(mu), _scalar(sigma)
        op = ny.rbf_operator(points, sig_f)
        f = ny.nys_sketch(op, ell, seed=seed, precision=precision)
        alpha, res, _ = ny.pcg_solve(op, f, mu_f, b.detach().contiguous(), tol=tol,
                                     precision=precision)
        if res[0].status != ny.NYS_OK:
            raise ny.NysError(res[0].status, "KRRSolve forward")
        ctx.op, ctx.f, ctx.mu, ctx.sigma = op, f, mu_f, sig_f
        ctx.precision, ctx.tol = precision, tol
        ctx.points = points
        ctx.save_for_backward(alpha)
        return alpha

    @staticmethod
    def backward(ctx, g):
        (alpha,) = ctx.saved_tensors
        # adjoint solve with the forward preconditioner (the matrix is symmetric)
        lam, res, _ = ny.pcg_solve(ctx.op, ctx.f, ctx.mu, g.detach().contiguous(), tol=ctx.tol,
                                   precision=ctx.precision)
        if res[0].status != ny.NYS_OK:
            raise ny.NysError(res[0].status, "KRRSolve adjoint")
        grad_b = lam
        grad_mu = -(lam @ alpha)
        dK_alpha = ny.nys_rbf_cross_matvec(ctx.points, ctx.points, ctx.sigma, alpha, kind=1)
        grad_sigma = -(lam @ dK_alpha)
        ctx.f.free()
        return grad_b, grad_mu.reshape(()), grad_sigma.reshape(()), None, None, None, None, None


class RBFCross(torch.autograd.Function):
    """pred = K(targets, points) alpha."""

    @staticmethod
    def forward(ctx, alpha, sigma, targets, points):
        sig_f = _scalar(sigma)
        ctx.sigma, ctx.targets, ctx.points = sig_f, targets, points
        ctx.save_for_backward(alpha)
        return ny.nys_rbf_cross_matvec(targets, points, sig_f, alpha.detach().contiguous(), kind=0)

    @staticmethod
    def backward(ctx, g):
        (alpha,) = ctx.saved_tensors
        g = g.detach().contiguous()
        grad_alpha = ny.nys_rbf_cross_matvec(ctx.points, ctx.targets, ctx.sigma, g, kind=0)
        dKv_alpha = ny.nys_rbf_cross_matvec(ctx.targets, ctx.points, ctx.sigma, alpha, kind=1)
        grad_sigma = g @ dKv_alpha
        return grad_alpha, grad_sigma.reshape(()), None, None


def validation_loss(points: torch.Tensor, y: torch.Tensor, vpoints: torch.Tensor,
                    yv: torch.Tensor, sigma: torch.Tensor, mu: torch.Tensor, ell: int,
                    precision: int = ny.NYS_PREC_MIXED, tol: float = 1e-10, seed: int = 0):
    """Mean squared validation error of KRR trained on (points, y); differentiable in
    y, mu and sigma (0-dim FP64 CUDA tensors)."""
    alpha = KRRSolve.apply(y, mu, sigma, points, ell, precision, tol, seed)
    pred = RBFCross.apply(alpha, sigma, vpoints, points)
    return torch.mean((pred - yv) ** 2)
