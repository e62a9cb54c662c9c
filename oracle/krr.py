"""Kernel ridge regression validation loss and its gradient (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

KRR (Sec. 6.5, Eq. (6.3)) solves (K + mu I) alpha = y for the training
targets y, with K the Gaussian kernel on the training points and mu the
diagonal shift (the paper's n*mu).  Predictions on validation points are
K_v alpha, (K_v)_ij = exp(-||t_i - x_j||^2 / (2 sigma^2)).

The paper does not differentiate the solve; the gradient below is plain
implicit differentiation (an adjoint solve with the same symmetric matrix):

  L        = mean((K_v alpha - y_v)^2)
  g        = (2/m) (K_v alpha - y_v)                 m = number of validation points
  lambda   = (K + mu I)^{-1} K_v^T g                 adjoint solve
  dL/dy    = lambda                                  (y is the right-hand side b)
  dL/dmu   = -lambda^T alpha
  dL/dsig  = g^T (dK_v/dsig) alpha - lambda^T (dK/dsig) alpha,
             dK_ij/dsig = K_ij ||x_i - x_j||^2 / sigma^3.

``solve(rhs)`` is any solver for (K + mu I) z = rhs; the tests pass the
dense Cholesky solve or Algorithm 3.
"""

from __future__ import annotations

import numpy as np

from . import operators as ops


def krr_loss(points, y, vpoints, yv, sigma: float, mu: float, solve=None):
    P = np.asarray(points, dtype=np.float64)
    if solve is None:
        K = ops.rbf_block(P, P, sigma)
        alpha = np.linalg.solve(K + mu * np.eye(P.shape[0]), y)
    else:
        alpha = solve(np.asarray(y, dtype=np.float64))
    pred = ops.rbf_cross_matmat(vpoints, P, sigma, alpha)
    return float(np.mean((pred - yv) ** 2)), alpha


def krr_loss_and_grads(points, y, vpoints, yv, sigma: float, mu: float, solve):
    """Returns dict(loss, alpha, lam, dL_db, dL_dmu, dL_dsigma)."""
    y = np.asarray(y, dtype=np.float64)
    yv = np.asarray(yv, dtype=np.float64)
    alpha = solve(y)
    pred = ops.rbf_cross_matmat(vpoints, points, sigma, alpha)
    resid = pred - yv
    m = yv.shape[0]
    loss = float(np.mean(resid ** 2))
    g = (2.0 / m) * resid
    # K_v^T g: rows of the cross kernel are validation points
    Kv_T_g = ops.rbf_cross_matmat(points, vpoints, sigma, g)
    lam = solve(Kv_T_g)
    dL_dmu = -float(lam @ alpha)
    dKv_alpha = ops.rbf_dsigma_matmat(points, sigma, alpha, targets=vpoints)
    dK_alpha = ops.rbf_dsigma_matmat(points, sigma, alpha)
    dL_dsigma = float(g @ dKv_alpha - lam @ dK_alpha)
    return dict(loss=loss, alpha=alpha, lam=lam, dL_db=lam, dL_dmu=dL_dmu, dL_dsigma=dL_dsigma)
