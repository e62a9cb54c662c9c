"""Regularization path with warm starts and factor reuse, plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's regularization-path experiments (Sec. 6.2 and the experimental
details of its appendix) solve (A + mu I) x = b for a decreasing sequence of
shifts: the first solve starts from zero and each later one from the previous
solution; the Nystrom factor is kept until the latest Algorithm 4 estimate of
||A - A_nys|| exceeds the error tolerance of the new shift, and a rebuilt
factor comes from Algorithm 5 started at twice the previous sketch size.
Readings:
* the error tolerance of shift mu is ``err_factor * mu`` (the experiments use
  30 mu) and Algorithm 5 runs Strategy 1 with that tolerance and q power steps;
* shifts are processed in decreasing order whatever order they are given in;
  results come back in the given order;
* once a factor reaches ell_max no later rebuild can enlarge it, so it is
  kept for the rest of the path (its estimate is then not defined);
* the r-th factor build draws its Gaussian test matrix and its power-step
  starts from ``draws(r)`` -- inputs, as everywhere in the oracle;
* each solve is Algorithm 3 with the per-shift iteration cap (500 in the
  experiments).
"""

from __future__ import annotations

import numpy as np

from . import nystrom as ny
from . import pcg


def regularization_path(matmat, n: int, mus, b: np.ndarray, ell0: int, ell_max: int,
                        err_factor: float, q: int, tol: float, maxit: int, draws):
    """``matmat(V)`` applies A to the columns of V; ``draws(r)`` returns the
    (Omega_raw n x ell_max, G [kmax][n]) of the r-th factor build.

    Returns a list (in the order of ``mus``) of dicts with x, iterations,
    status, ell, resketched, E (the estimate in force), the factor (U, lam)
    used, and the number of builds."""
    mus = [float(m) for m in mus]
    order = sorted(range(len(mus)), key=lambda i: -mus[i])
    b = np.asarray(b, dtype=np.float64)
    x = None
    fac = None
    E = float("inf")
    capped = False
    builds = 0
    out = [None] * len(mus)
    for idx in order:
        mu = mus[idx]
        tol_E = err_factor * mu
        rebuilt = False
        if fac is None or (not capped and not (E <= tol_E)):
            start = ell0 if fac is None else min(2 * fac["ell"], ell_max)
            Om, G = draws(builds)
            builds += 1
            fac = ny.adaptive_nystrom(matmat, n, start, ell_max, tol_E, q, Om, G, rule="err")
            E = fac["E"]
            capped = fac["ell"] >= ell_max
            rebuilt = True
        U, lam = fac["U"], fac["lam"]
        sol = pcg.nys_pcg(lambda v: matmat(v[:, None])[:, 0], mu, b, x,
                          lambda r: ny.precond_inverse_apply(U, lam, mu, r), tol, maxit)
        x = sol["x"]
        out[idx] = dict(x=x.copy(), iterations=sol["iterations"], status=sol["status"],
                        ell=fac["ell"], resketched=rebuilt, E=E, U=U, lam=lam)
    return out, builds
