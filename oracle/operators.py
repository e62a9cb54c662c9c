"""Matvec oracles x -> A x for the three operators of the hot path (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper accesses A only through matvecs (Sec. 1.1).  The three operators:

* dense:  A given explicitly (n x n, symmetric psd).
* gram:   A = X^T X for a data matrix X (m x n), the ridge-regression normal
          operator of Eq. (1.7) with the 1/n factor folded into X.  Applied
          matrix-free as X^T (X v); X is upcast to FP64 first.
* rbf:    A = K with K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)), the Gaussian
          kernel of Sec. 6.5 (Eq. (6.3) adds the shift).  Squared distances are
          summed directly as sum_k (x_ik - x_jk)^2, never by the norm expansion,
          so they carry no cancellation error.

Every ``*_matmat`` applies A (without the shift mu) to the columns of V.
Passing ``dtype=np.float32`` gives the float32 emulation used by the
refinement oracle (all arithmetic in numpy float32).
"""

from __future__ import annotations

import numpy as np


def dense_matmat(A: np.ndarray, V: np.ndarray, dtype=np.float64) -> np.ndarray:
    return np.asarray(A, dtype=dtype) @ np.asarray(V, dtype=dtype)


def gram_matmat(X: np.ndarray, V: np.ndarray, dtype=np.float64) -> np.ndarray:
    Xd = np.asarray(X, dtype=dtype)
    Vd = np.asarray(V, dtype=dtype)
    return Xd.T @ (Xd @ Vd)


def sq_dists(P: np.ndarray, Q: np.ndarray, dtype=np.float64) -> np.ndarray:
    """D_ij = sum_k (p_ik - q_jk)^2, summed term by term."""
    P = np.asarray(P, dtype=dtype)
    Q = np.asarray(Q, dtype=dtype)
    D = np.zeros((P.shape[0], Q.shape[0]), dtype=dtype)
    for k in range(P.shape[1]):
        diff = P[:, k][:, None] - Q[:, k][None, :]
        D += diff * diff
    return D


def rbf_block(P: np.ndarray, Q: np.ndarray, sigma: float, dtype=np.float64) -> np.ndarray:
    """Kernel block K_ij = exp(-||p_i - q_j||^2 / (2 sigma^2))."""
    D = sq_dists(P, Q, dtype)
    return np.exp(-D / dtype(2.0 * sigma * sigma))


def rbf_matmat(points: np.ndarray, sigma: float, V: np.ndarray, dtype=np.float64,
               row_chunk: int = 512, cols: np.ndarray | None = None) -> np.ndarray:
    """K V with K formed block by block (rows in chunks), never stored whole.

    ``cols`` (optional) restricts the output to those rows of K V, for sampled
    checks at sizes where the full product is too slow."""
    P = np.asarray(points, dtype=dtype)
    Vd = np.asarray(V, dtype=dtype)
    rows = np.arange(P.shape[0]) if cols is None else np.asarray(cols)
    out = np.empty((rows.shape[0],) + Vd.shape[1:], dtype=dtype)
    for r0 in range(0, rows.shape[0], row_chunk):
        r = rows[r0:r0 + row_chunk]
        Kb = rbf_block(P[r], P, sigma, dtype)
        out[r0:r0 + r.shape[0]] = Kb @ Vd
    return out


def rbf_dsigma_matmat(points: np.ndarray, sigma: float, V: np.ndarray, row_chunk: int = 512,
                      targets: np.ndarray | None = None) -> np.ndarray:
    """(dK/dsigma) V with dK_ij/dsigma = K_ij * D_ij / sigma^3 (D squared distance).

    With ``targets`` given, the rows are the kernel between ``targets`` and
    ``points`` (a cross kernel), else K is the square kernel on ``points``."""
    P = np.asarray(points, dtype=np.float64)
    T = P if targets is None else np.asarray(targets, dtype=np.float64)
    Vd = np.asarray(V, dtype=np.float64)
    out = np.empty((T.shape[0],) + Vd.shape[1:])
    for r0 in range(0, T.shape[0], row_chunk):
        D = sq_dists(T[r0:r0 + row_chunk], P)
        Kb = np.exp(-D / (2.0 * sigma * sigma))
        out[r0:r0 + D.shape[0]] = (Kb * D / sigma ** 3) @ Vd
    return out


def rbf_cross_matmat(targets: np.ndarray, points: np.ndarray, sigma: float, V: np.ndarray,
                     row_chunk: int = 512) -> np.ndarray:
    """K_v V with (K_v)_ij = exp(-||t_i - x_j||^2 / (2 sigma^2)) (prediction kernel)."""
    T = np.asarray(targets, dtype=np.float64)
    P = np.asarray(points, dtype=np.float64)
    Vd = np.asarray(V, dtype=np.float64)
    out = np.empty((T.shape[0],) + Vd.shape[1:])
    for r0 in range(0, T.shape[0], row_chunk):
        out[r0:r0 + min(row_chunk, T.shape[0] - r0)] = rbf_block(T[r0:r0 + row_chunk], P, sigma) @ Vd
    return out


class Operator:
    """Bundles one of the three operators with its apply function."""

    def __init__(self, kind: str, data: np.ndarray, sigma: float = 0.0):
        assert kind in ("dense", "gram", "rbf")
        self.kind = kind
        self.data = data
        self.sigma = float(sigma)
        if kind == "dense":
            self.n = data.shape[0]
        elif kind == "gram":
            self.n = data.shape[1]
        else:
            self.n = data.shape[0]

    def matmat(self, V: np.ndarray, dtype=np.float64) -> np.ndarray:
        if self.kind == "dense":
            return dense_matmat(self.data, V, dtype)
        if self.kind == "gram":
            return gram_matmat(self.data, V, dtype)
        return rbf_matmat(self.data, self.sigma, V, dtype)

    def explicit(self) -> np.ndarray:
        """The n x n matrix A itself (small n only)."""
        if self.kind == "dense":
            return np.asarray(self.data, dtype=np.float64)
        if self.kind == "gram":
            X = np.asarray(self.data, dtype=np.float64)
            return X.T @ X
        return rbf_block(self.data, self.data, self.sigma)
