"""Nystrom PCG (Algorithm 3), its independent-batch form and FP64-residual
iterative refinement, plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 3 (Sec. 5.2) is left-preconditioned CG.  Readings:
* the loop test of Algorithm 3 compares ||r||_2 with an absolute eta; the
  target here is relative: stop as soon as the recurrence residual satisfies
  ||r_t||_2 <= tol * ||b||_2, tested before the first iteration as well;
* ``iterations`` counts the A-matvecs made inside the loop (r_0 costs one
  more when x_0 != 0);
* the symbol v_0 in the step-size formula of Algorithm 3 is the v just
  computed;
* the iteration cap is ``maxit`` (500 in the paper's experiments, Sec. 6.2);
* a non-positive or non-finite p^T v stops the loop with status "breakdown".

Batched solves (many mu values and right-hand sides sharing one factor) are
independent recurrences, so the oracle is a loop of single solves.

Iterative refinement (not in the paper): an FP64 outer loop
    r = b - (A + mu I) x   (FP64),  stop if ||r|| <= tol ||b||,
    d = PCG on (A + mu I) d = r in float32 to relative tolerance inner_tol,
    x = x + d.
"""

from __future__ import annotations

import numpy as np

CONVERGED, MAXIT, BREAKDOWN = "converged", "maxit", "breakdown"


def nys_pcg(matvec, mu: float, b: np.ndarray, x0: np.ndarray | None, precond_inv, tol: float,
            maxit: int = 500, dtype=np.float64):
    """Algorithm 3.  ``matvec(v)`` applies A (no shift), ``precond_inv(r)``
    applies P^{-1} (identity gives textbook CG).

    With dtype=float32 the vectors and the matvec run in float32 while the
    scalar recurrences (dot products, alpha, beta) run in float64.

    Returns dict(x, iterations, status, res_hist)."""
    f = dtype
    b = np.asarray(b, dtype=f)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=f).copy()

    def dot(a, c):
        return float(np.dot(a.astype(np.float64), c.astype(np.float64)))

    def amu(v):
        return (np.asarray(matvec(v), dtype=f) + f(mu) * v).astype(f)

    r = (b - amu(x)).astype(f) if x0 is not None else b.copy()
    z = np.asarray(precond_inv(r), dtype=f)
    p = z.copy()
    rz = dot(r, z)
    thresh = tol * np.sqrt(dot(b, b))
    rnorm = np.sqrt(dot(r, r))
    hist = [rnorm]
    it = 0
    status = CONVERGED
    while rnorm > thresh:
        if it >= maxit:
            status = MAXIT
            break
        v = amu(p)
        pv = dot(p, v)
        if not np.isfinite(pv) or pv <= 0.0:
            status = BREAKDOWN
            break
        alpha = rz / pv
        x = (x + f(alpha) * p).astype(f)
        r = (r - f(alpha) * v).astype(f)
        z = np.asarray(precond_inv(r), dtype=f)
        rz_new = dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = (z + f(beta) * p).astype(f)
        it += 1
        rnorm = np.sqrt(dot(r, r))
        hist.append(rnorm)
    return dict(x=x, iterations=it, status=status, res_hist=np.array(hist))


def batched_pcg(matvec, mus, B: np.ndarray, precond_inv_for_mu, tol: float, maxit: int = 500):
    """Independent solves (A + mu_s I) x_s = b_s for the columns s of B
    ([nsys][n]); ``precond_inv_for_mu(mu)`` returns the P^{-1} apply for that
    shift.  Each column is exactly its own single solve."""
    out = []
    for s in range(B.shape[0]):
        mu = float(mus[s])
        out.append(nys_pcg(matvec, mu, B[s], None, precond_inv_for_mu(mu), tol, maxit))
    return out


def refine_solve(matvec_hi, matvec_lo, precond_inv_lo, mu: float, b: np.ndarray, tol: float,
                 inner_tol: float, maxit: int = 500, max_refine: int = 20):
    """FP64-residual iterative refinement around a float32 PCG.

    ``matvec_hi`` applies A in FP64, ``matvec_lo`` and ``precond_inv_lo``
    work on float32 vectors.  Returns dict(x, outer, inner_iterations,
    status, true_res_hist)."""
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = []
    inner_total = 0
    status = MAXIT
    for k in range(max_refine + 1):
        r = b - (matvec_hi(x) + mu * x)
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= tol:
            status = CONVERGED
            break
        if k == max_refine or inner_total >= maxit:
            break
        # maxit bounds the inner iterations summed over all refinement steps
        inner = nys_pcg(matvec_lo, mu, r.astype(np.float32), None, precond_inv_lo, inner_tol,
                        maxit - inner_total, dtype=np.float32)
        inner_total += inner["iterations"]
        x = x + inner["x"].astype(np.float64)
    return dict(x=x, outer=len(hist) - 1, inner_iterations=inner_total, status=status,
                true_res_hist=np.array(hist))


def direct_solve(A: np.ndarray, mu: float, b: np.ndarray) -> np.ndarray:
    """x_star = (A + mu I)^{-1} b by dense Cholesky (the plain definition)."""
    import scipy.linalg as sla
    n = A.shape[0]
    c = sla.cho_factor(A + mu * np.eye(n))
    return sla.cho_solve(c, b)
