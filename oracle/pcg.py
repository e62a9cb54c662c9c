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

Block PCG (Sec. 5.2, "Block Nystrom PCG"): O'Leary's block CG for several
right-hand sides of one shifted matrix, with the preconditioner of Eq. (5.3)
and the orthogonalisation pre-processing of Feng, Owen & Peric (1995).  The
paper names the two ingredients only; the readings here are:
* pre-processing: the initial residual block is factored R_0 = Q S (thin QR),
  block CG runs on (A + mu I) Y = Q from Y = 0, and X = X_0 + Y S;
* the recurrence is O'Leary's with the scaling matrices gamma_k = I:
  alpha = (P^T V)^{-1} (Z^T R), beta = (Z^T R)^{-1} (Z_new^T R_new), both s x s
  solves by Cholesky of the symmetrised left factor;
* column j stops being a target when ||(R S) e_j|| <= tol ||b_j|| (its
  recurrence residual in the original scaling); the loop runs until every
  column meets it, tested before the first iteration as well; a column that
  meets it at the start (b_j = 0 included) leaves the block;
* ``iterations`` counts block products (A + mu I) P; a failed Cholesky or a
  non-finite value stops the loop with status "breakdown" for the columns not
  yet converged.

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


def block_pcg(matmat, mu: float, B: np.ndarray, X0: np.ndarray | None, precond_inv, tol: float,
              maxit: int = 500):
    """Block Nystrom PCG (readings in the module docstring).  ``B`` and ``X0``
    are [s][n] (system-major); ``matmat(V)`` applies A to the columns of the
    n x k matrix V, ``precond_inv(V)`` applies P^{-1} to them.

    Returns dict(X [s][n], iterations, status [s], rel_res [s], res_hist
    (iterations+1) x s)."""
    import scipy.linalg as sla
    Bc = np.asarray(B, dtype=np.float64).T.copy()
    n, s = Bc.shape
    X = np.zeros_like(Bc) if X0 is None else np.asarray(X0, dtype=np.float64).T.copy()

    def amu(V):
        return np.asarray(matmat(V), dtype=np.float64) + mu * V

    R0 = Bc - amu(X) if X0 is not None else Bc.copy()
    thresh = tol * np.linalg.norm(Bc, axis=0)
    res = np.linalg.norm(R0, axis=0)
    status = [CONVERGED] * s
    act = np.nonzero(res > thresh)[0]
    hist = [res.copy()]
    it = 0
    if act.size:
        Q, S = np.linalg.qr(R0[:, act])          # pre-processing: R_0 = Q S
        Y = np.zeros((n, act.size))
        R = Q
        Z = np.asarray(precond_inv(R), dtype=np.float64)
        P = Z.copy()
        rho = Z.T @ R
        broke = False
        while True:
            res[act] = np.linalg.norm(R @ S, axis=0)
            if it > 0:
                hist.append(res.copy())
            if np.all(res[act] <= thresh[act]) or it >= maxit or broke:
                break
            V = amu(P)
            G = P.T @ V
            try:
                alpha = sla.cho_solve(sla.cho_factor(0.5 * (G + G.T)), rho)
            except (np.linalg.LinAlgError, ValueError):
                broke = True
                break
            Y = Y + P @ alpha
            R = R - V @ alpha
            Z = np.asarray(precond_inv(R), dtype=np.float64)
            rho_new = Z.T @ R
            it += 1
            try:
                beta = sla.cho_solve(sla.cho_factor(0.5 * (rho + rho.T)), rho_new)
            except (np.linalg.LinAlgError, ValueError):
                broke = True        # this step stands; the next one cannot be formed
                continue
            P = Z + P @ beta
            rho = rho_new
            if not np.all(np.isfinite(P)):
                broke = True
        X[:, act] = X[:, act] + Y @ S
        for j in act:
            if not res[j] <= thresh[j]:
                status[j] = BREAKDOWN if broke else MAXIT
    bn = np.linalg.norm(Bc, axis=0)
    rel = np.where(bn > 0, res / np.where(bn > 0, bn, 1.0), res)
    return dict(X=X.T.copy(), iterations=it, status=status, rel_res=rel, res_hist=np.array(hist))


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


def cg_rate(kappa: float) -> float:
    """Per-iteration contraction of the CG error in the energy norm for a
    system of condition number kappa, (sqrt(kappa) - 1) / (sqrt(kappa) + 1):
    the standard CG bound behind the convergence corollaries of Sec. 1 and
    Sec. 5.3 (delta_t < 2 rate^t)."""
    r = float(np.sqrt(kappa))
    return (r - 1.0) / (r + 1.0)


def iterations_to(rate: float, eps: float) -> int:
    """Smallest t with 2 rate^t <= eps: ceil(log(2/eps) / log(1/rate))."""
    return int(np.ceil(np.log(2.0 / eps) / np.log(1.0 / rate)))


def direct_solve(A: np.ndarray, mu: float, b: np.ndarray) -> np.ndarray:
    """x_star = (A + mu I)^{-1} b by dense Cholesky (the plain definition)."""
    import scipy.linalg as sla
    n = A.shape[0]
    c = sla.cho_factor(A + mu * np.eye(n))
    return sla.cho_solve(c, b)
