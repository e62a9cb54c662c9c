"""Randomized Nystrom approximation and preconditioner, plain FP64 (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows, step by step and in the paper's order:
* Algorithm 1 (Sec. 2.2): randomized Nystrom approximation A_nys = U Lam U^T;
* Eq. (5.3) (Sec. 5.1.2): the Nystrom preconditioner P and its inverse;
* Algorithm 4 (App. E.1): randomized power estimate of ||E||, E = A - A_nys;
* Algorithm 5 (App. E.2) with Strategy 1 (Sec. 5.4.1) and Strategy 2
  (Sec. 5.4.2): adaptive rank doubling reusing Omega and Y;
* Algorithm 2 with Eq. (4.1) (Sec. 4): Nystrom sketch-and-solve.

Readings where the paper is loose (all listed in the design notes):
* eps(x) is MATLAB's spacing of floating-point numbers at |x|,
  2^(floor(log2|x|) - p) with p = 52 for double (p = 23 for a float32 sketch).
* Omega^T Y_nu is symmetric only up to rounding; it is symmetrised before the
  Cholesky factorisation (MATLAB's chol reads one triangle).
* B = Y_nu / C is MATLAB right division: B = Y_nu C^{-1}, C upper triangular
  with C^T C = Omega^T Y_nu.
* If the Cholesky factorisation fails, nu is multiplied by 10 and the shift
  redone, at most 6 times; after that the approximation is reported not psd.
* Lam is returned in descending order; lam_hat_ell is its last entry.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

MAX_SHIFT_ESCALATIONS = 6


class NotPSDError(RuntimeError):
    pass


def eps_spacing(x: float, mantissa_bits: int = 52) -> float:
    """MATLAB eps(x): spacing of floating-point numbers at |x| (x finite, != 0).

    For a double, eps(x) = 2^(e - 52) where 2^e <= |x| < 2^(e+1)."""
    ax = abs(float(x))
    if ax == 0.0:
        return 2.0 ** -1074 if mantissa_bits == 52 else 2.0 ** -149
    _, e2 = math.frexp(ax)          # ax = f * 2^e2, f in [0.5, 1)
    return math.ldexp(1.0, (e2 - 1) - mantissa_bits)


def thin_qr(Omega: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Omega): the Q of a thin QR (Alg. 1, step 2)."""
    Q, _ = np.linalg.qr(np.asarray(Omega, dtype=np.float64), mode="reduced")
    return Q


def shifted_core(Q: np.ndarray, Y: np.ndarray, nu: float):
    """Steps 4-9 of Algorithm 1 given the test matrix Q and the sketch Y = A Q.

    Returns (U, lam, nu_used, escalations)."""
    nu_used = float(nu)
    for esc in range(MAX_SHIFT_ESCALATIONS + 1):
        Ynu = Y + nu_used * Q                         # shift for stability
        M = Q.T @ Ynu
        M = 0.5 * (M + M.T)
        try:
            L = np.linalg.cholesky(M)                 # M = L L^T, C = L^T
        except np.linalg.LinAlgError:
            nu_used *= 10.0
            continue
        C = L.T
        # B = Ynu C^{-1}  <=>  C^T B^T = Ynu^T
        B = sla.solve_triangular(C, Ynu.T, trans="T", lower=False).T
        U, S, _ = np.linalg.svd(B, full_matrices=False)   # thin SVD
        lam = np.maximum(0.0, S * S - nu_used)            # remove shift
        return U, lam, nu_used, esc
    raise NotPSDError("Cholesky of Omega^T Y_nu failed after shift escalation")


def rand_nystrom(matmat, Omega_raw: np.ndarray, mantissa_bits: int = 52):
    """Algorithm 1.  ``matmat(V)`` applies A to the columns of V; ``Omega_raw``
    is the Gaussian test matrix (n x ell) of step 1, passed in.

    Returns a dict with U (n x ell), lam (ell, descending), nu, Q, Y."""
    Q = thin_qr(Omega_raw)                                  # step 2
    Y = np.asarray(matmat(Q), dtype=np.float64)             # step 3: ell matvecs
    nu = eps_spacing(np.linalg.norm(Y, "fro"), mantissa_bits)   # step 4
    U, lam, nu_used, esc = shifted_core(Q, Y, nu)           # steps 5-9
    return dict(U=U, lam=lam, nu=nu_used, nu0=nu, escalations=esc, Q=Q, Y=Y)


# ---------------------------------------------------------------------------
# Preconditioner, Eq. (5.3)
# ---------------------------------------------------------------------------

def precond_inverse_apply(U: np.ndarray, lam: np.ndarray, mu: float, V: np.ndarray) -> np.ndarray:
    """P^{-1} V = (lam_ell + mu) U (Lam + mu I)^{-1} U^T V + (I - U U^T) V."""
    V = np.asarray(V, dtype=np.float64)
    if U.shape[1] == 0:
        return V.copy()
    lam_ell = lam[-1]
    W = U.T @ V
    scale = (lam_ell + mu) / (lam + mu)
    term1 = U @ (scale[:, None] * W) if W.ndim == 2 else U @ (scale * W)
    return term1 + V - U @ W


def precond_apply(U: np.ndarray, lam: np.ndarray, mu: float, V: np.ndarray) -> np.ndarray:
    """P V = (lam_ell + mu)^{-1} U (Lam + mu I) U^T V + (I - U U^T) V."""
    V = np.asarray(V, dtype=np.float64)
    lam_ell = lam[-1]
    W = U.T @ V
    scale = (lam + mu) / (lam_ell + mu)
    term1 = U @ (scale[:, None] * W) if W.ndim == 2 else U @ (scale * W)
    return term1 + V - U @ W


def precond_inverse_apply_f32(U32: np.ndarray, lam: np.ndarray, mu: float, v32: np.ndarray) -> np.ndarray:
    """Float32 emulation of Eq. (5.3) for the refinement oracle: U and the
    vector in float32, the ell coefficients in float64 then rounded."""
    w = (U32.T @ v32).astype(np.float64)
    coef = ((lam[-1] + mu) / (lam + mu) - 1.0) * w
    return (v32 + U32 @ coef.astype(np.float32)).astype(np.float32)


# ---------------------------------------------------------------------------
# Algorithm 4: randomized power method for ||E||
# ---------------------------------------------------------------------------

def power_error_estimate(matvec, U: np.ndarray, lam: np.ndarray, g: np.ndarray, q: int) -> float:
    """``matvec(v)`` applies A (no shift); ``g`` is the Gaussian start of step 1."""
    v0 = np.asarray(g, dtype=np.float64) / np.linalg.norm(g)
    E = 0.0
    for _ in range(q):
        v = matvec(v0) - U @ (lam * (U.T @ v0))
        E = float(v0 @ v)
        v = v / np.linalg.norm(v)
        v0 = v
    return E


# ---------------------------------------------------------------------------
# Algorithm 5: adaptive rank doubling (Strategy 1), ratio rule (Strategy 2)
# ---------------------------------------------------------------------------

def adaptive_nystrom(matmat, n: int, ell0: int, ell_max: int, tol: float, q: int,
                     Omega_raw: np.ndarray, G: np.ndarray | None, rule: str = "err",
                     mu: float | None = None, lambda_rule: bool = False,
                     mantissa_bits: int = 52):
    """Algorithm 5.  The k-th Gaussian block of step 4 is the next ``m``
    columns of ``Omega_raw`` (n x ell_max); the k-th error estimate starts
    from ``G[k]``.

    rule = "err":   stop when the Algorithm 4 estimate E <= tol (Strategy 1);
                    with ``lambda_rule`` also require lam_ell <= tol / 11.
    rule = "ratio": stop when lam_ell / mu <= tol (Strategy 2); no estimate.

    Returns a dict with U, lam, nu, ell, E (last estimate or nan), the
    number of doublings and the per-step history."""
    assert rule in ("err", "ratio")
    if rule == "ratio":
        assert mu is not None and mu > 0
    Qs, Ys = [], []
    ell_tot = 0
    ell_next = min(ell0, ell_max)   # "ell_0" of the pseudocode: total after the next block
    m = ell_next                    # size of the next block
    k_est = 0
    history = []
    E = float("nan")
    U = lam = None
    nu = 0.0

    def add_block(mm):
        nonlocal ell_tot
        Om0 = Omega_raw[:, ell_tot:ell_tot + mm]
        Q0 = thin_qr(Om0)
        Y0 = np.asarray(matmat(Q0), dtype=np.float64)
        Qs.append(Q0)
        Ys.append(Y0)
        ell_tot += mm

    def core():
        Q = np.concatenate(Qs, axis=1)
        Y = np.concatenate(Ys, axis=1)
        nu0 = math.sqrt(n) * eps_spacing(np.linalg.norm(Y, 2), mantissa_bits)
        return shifted_core(Q, Y, nu0)

    while True:
        add_block(m)
        U, lam, nu, _ = core()
        if rule == "err":
            E = power_error_estimate(lambda v: matmat(v[:, None])[:, 0], U, lam, G[k_est], q)
            k_est += 1
            stop = E <= tol and (not lambda_rule or lam[-1] <= tol / 11.0)
        else:
            stop = lam[-1] / mu <= tol
        history.append(dict(ell=ell_tot, E=E, lam_ell=float(lam[-1]), nu=nu))
        if stop:
            break
        m = ell_next
        ell_next = 2 * ell_next
        if ell_next > ell_max:
            ell_next = ell_next - m
            m = ell_max - ell_next
            if m > 0:
                add_block(m)
                U, lam, nu, _ = core()
                E = float("nan")
                history.append(dict(ell=ell_tot, E=E, lam_ell=float(lam[-1]), nu=nu))
            break
    return dict(U=U, lam=lam, nu=nu, ell=ell_tot, E=E, history=history,
                doublings=len(history) - 1)


def adaptive_tau0(tau: float) -> float:
    """Theorem 5.6 (3): with the error tolerance tau mu of Algorithm 5, PCG
    contracts by tau0 = (sqrt(1 + 12 tau / 11) - 1) / (sqrt(1 + 12 tau / 11) + 1)
    per iteration."""
    r = math.sqrt(1.0 + 12.0 * tau / 11.0)
    return (r - 1.0) / (r + 1.0)


def kappa_estimate(lam_ell: float, mu: float, E: float) -> float:
    """Posterior bound of Eq. (5.6): kappa <= (lam_ell + mu + ||E||) / mu."""
    return (lam_ell + mu + E) / mu


# ---------------------------------------------------------------------------
# Algorithm 2: Nystrom sketch-and-solve via Eq. (4.1)
# ---------------------------------------------------------------------------

def sketch_and_solve(U: np.ndarray, lam: np.ndarray, mu: float, b: np.ndarray) -> np.ndarray:
    """x = U (Lam + mu I)^{-1} U^T b + (1/mu)(b - U U^T b)."""
    w = U.T @ b
    return U @ (w / (lam + mu)) + (b - U @ w) / mu


# ---------------------------------------------------------------------------
# Brute-force helpers for the pins (small n only)
# ---------------------------------------------------------------------------

def preconditioned_spectrum(A: np.ndarray, U: np.ndarray, lam: np.ndarray, mu: float) -> np.ndarray:
    """Eigenvalues of P^{-1/2} A_mu P^{-1/2} (ascending), by dense algebra."""
    n = A.shape[0]
    Pinv = precond_inverse_apply(U, lam, mu, np.eye(n))
    Pinv = 0.5 * (Pinv + Pinv.T)
    w, V = np.linalg.eigh(Pinv)
    S = (V * np.sqrt(np.maximum(w, 0.0))) @ V.T
    M = S @ (A + mu * np.eye(n)) @ S
    return np.linalg.eigvalsh(0.5 * (M + M.T))


def effective_dimension(eigs: np.ndarray, mu: float) -> float:
    """d_eff(mu) = sum_j lam_j / (lam_j + mu), Eq. (1.4)."""
    eigs = np.asarray(eigs, dtype=np.float64)
    return float(np.sum(eigs / (eigs + mu)))
