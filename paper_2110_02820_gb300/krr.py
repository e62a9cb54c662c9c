"""Differentiable kernel ridge regression on the Nystrom PCG library.

The training system (K + mu I) alpha = b (Sec. 6.5, Eq. (6.3), with mu the
diagonal actually added) is solved by Nystrom PCG; its gradient comes from one
more solve with the same matrix (the adjoint), preconditioned by the same
Nystrom factor:

    lambda     = (K + mu I)^{-1} dL/dalpha
    dL/db      = lambda
    dL/dmu     = -lambda^T alpha
    dL/dsigma  = -lambda^T (dK/dsigma) alpha (+ g^T (dK_v/dsigma) alpha for the
                 validation objective),  dK_ij/dsigma = K_ij ||x_i-x_j||^2 / sigma^3

The solves, the products with K, K_v and their sigma-derivatives, the
objective and every dot product run in the CUDA library (nys_krr_validation,
nys_krr_gradients); this module only wires their outputs into
torch.autograd (and scales them by the incoming gradient).
"""

from __future__ import annotations

import torch

from . import nyspcg as ny


def _scalar(x) -> float:
    return float(x.detach().item()) if torch.is_tensor(x) else float(x)


def _solve(points, sig_f, mu_f, b, ell, precision, tol, seed):
    op = ny.rbf_operator(points, sig_f)
    f = ny.nys_sketch(op, ell, seed=seed, precision=precision)
    alpha, res, _ = ny.pcg_solve(op, f, mu_f, b.detach().contiguous(), tol=tol,
                                 precision=precision)
    if res[0].status != ny.NYS_OK:
        f.free()
        raise ny.NysError(res[0].status, "KRR training solve")
    return op, f, alpha


def _adjoint(op, f, mu_f, rhs, tol, precision):
    # adjoint solve with the forward preconditioner (the matrix is symmetric)
    lam, res, _ = ny.pcg_solve(op, f, mu_f, rhs.detach().contiguous(), tol=tol,
                               precision=precision)
    if res[0].status != ny.NYS_OK:
        raise ny.NysError(res[0].status, "KRR adjoint solve")
    return lam


class KRRSolve(torch.autograd.Function):
    """alpha = (K_sigma + mu I)^{-1} b with a Nystrom-preconditioned solve."""

    @staticmethod
    def forward(ctx, b, mu, sigma, points, ell, precision, tol, seed):
        mu_f, sig_f = _scalar(mu), _scalar(sigma)
        op, f, alpha = _solve(points, sig_f, mu_f, b, ell, precision, tol, seed)
        ctx.op, ctx.f, ctx.mu, ctx.sigma = op, f, mu_f, sig_f
        ctx.precision, ctx.tol = precision, tol
        ctx.points = points
        ctx.save_for_backward(alpha)
        return alpha

    @staticmethod
    def backward(ctx, g):
        (alpha,) = ctx.saved_tensors
        try:
            lam = _adjoint(ctx.op, ctx.f, ctx.mu, g, ctx.tol, ctx.precision)
            dmu, dsig = ny.nys_krr_gradients(ctx.points, None, ctx.sigma, alpha, lam, None)
        finally:
            ctx.f.free()
        one = torch.ones((), dtype=torch.float64, device=alpha.device)
        return lam, one * dmu, one * dsig, None, None, None, None, None


class KRRValidationLoss(torch.autograd.Function):
    """L = mean((K_v alpha - yv)^2), alpha = (K_sigma + mu I)^{-1} b."""

    @staticmethod
    def forward(ctx, b, mu, sigma, points, vpoints, yv, ell, precision, tol, seed):
        mu_f, sig_f = _scalar(mu), _scalar(sigma)
        op, f, alpha = _solve(points, sig_f, mu_f, b, ell, precision, tol, seed)
        loss, g, ktg = ny.nys_krr_validation(points, vpoints, sig_f, alpha, yv.detach().contiguous())
        ctx.op, ctx.f, ctx.mu, ctx.sigma = op, f, mu_f, sig_f
        ctx.precision, ctx.tol = precision, tol
        ctx.points, ctx.vpoints = points, vpoints
        ctx.save_for_backward(alpha, g, ktg)
        return torch.tensor(loss, dtype=torch.float64, device=alpha.device)

    @staticmethod
    def backward(ctx, gL):
        alpha, g, ktg = ctx.saved_tensors
        try:
            lam = _adjoint(ctx.op, ctx.f, ctx.mu, ktg, ctx.tol, ctx.precision)
            dmu, dsig = ny.nys_krr_gradients(ctx.points, ctx.vpoints, ctx.sigma, alpha, lam, g)
        finally:
            ctx.f.free()
        return (gL * lam, gL * dmu, gL * dsig, None, None, None, None, None, None, None)


def validation_loss(points: torch.Tensor, y: torch.Tensor, vpoints: torch.Tensor,
                    yv: torch.Tensor, sigma: torch.Tensor, mu: torch.Tensor, ell: int,
                    precision: int = ny.NYS_PREC_MIXED, tol: float = 1e-10, seed: int = 0):
    """Mean squared validation error of KRR trained on (points, y); differentiable in
    y, mu and sigma (0-dim FP64 CUDA tensors)."""
    return KRRValidationLoss.apply(y, mu, sigma, points, vpoints, yv, ell, precision, tol, seed)
