"""Seeded synthetic inputs for the Nystrom PCG workloads.

This module only draws inputs: test matrices, right-hand sides, data
matrices and point clouds.  It holds none of the method's arithmetic, so
that both the CUDA path (through the tests and the benchmark) and the CPU
oracle can take their inputs from it.

Every array comes from its own numpy ``PCG64`` stream keyed by
``(seed, stream_tag)``, so adding one array never shifts another.  Large
arrays are filled in row chunks, each chunk from a stream keyed by
``(seed, stream_tag, chunk)``; the chunks are drawn on a thread pool
(numpy releases the GIL inside bulk draws).

Workload shapes follow the paper's experiments (Sec. 6): ridge regression on
tall feature matrices whose column scales decay like random features, and
kernel ridge regression with a Gaussian kernel whose bandwidth sits at the
median pairwise distance (Sec. 6.3).
"""

from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

# Stream tags: one per kind of array.
S_OMEGA, S_B, S_Y, S_X, S_G, S_W, S_Q, S_MEANS, S_LABEL, S_NOISE, S_SUB, S_COLS = range(12)

_CHUNK_ROWS = 8192


def rng(seed: int, tag: int, chunk: int | None = None) -> np.random.Generator:
    key = [int(seed), int(tag)] if chunk is None else [int(seed), int(tag), int(chunk)]
    return np.random.Generator(np.random.PCG64(key))


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def gaussian(shape, seed: int, tag: int, dtype=np.float64) -> np.ndarray:
    """N(0,1) array; tall arrays are drawn in independent row chunks."""
    shape = tuple(int(s) for s in (shape if isinstance(shape, (tuple, list)) else (shape,)))
    rows = shape[0] if shape else 1
    if rows <= _CHUNK_ROWS:
        return rng(seed, tag).standard_normal(shape, dtype=np.float64).astype(dtype, copy=False)
    out = np.empty(shape, dtype=dtype)
    nchunks = (rows + _CHUNK_ROWS - 1) // _CHUNK_ROWS

    def fill(c):
        r0 = c * _CHUNK_ROWS
        r1 = min(rows, r0 + _CHUNK_ROWS)
        g = rng(seed, tag, c)
        if dtype == np.float32:
            out[r0:r1] = g.standard_normal((r1 - r0,) + shape[1:], dtype=np.float32)
        else:
            out[r0:r1] = g.standard_normal((r1 - r0,) + shape[1:], dtype=np.float64)

    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(fill, range(nchunks)))
    return out


# --------------------------------------------------------------------------
# Dense SPD test matrix with a prescribed spectrum (dense FP64 workload)
# --------------------------------------------------------------------------

def orthogonal(n: int, seed: int) -> np.ndarray:
    """Q factor of the QR of a seeded n x n N(0,1) matrix (signs fixed so
    that diag(R) > 0)."""
    G = gaussian((n, n), seed, S_Q)
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def power_spectrum(n: int, exponent: float = 1.5) -> np.ndarray:
    """lambda_i = (i+1)^-exponent for i = 0..n-1 (lambda_0 = 1)."""
    return (np.arange(n, dtype=np.float64) + 1.0) ** (-exponent)


def dense_spd(n: int, seed: int, eigenvalues: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """A = Q diag(lam) Q^T with Q from :func:`orthogonal`.  Returns (A, lam)."""
    lam = power_spectrum(n) if eigenvalues is None else np.asarray(eigenvalues, dtype=np.float64)
    Q = orthogonal(n, seed)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return A, lam


# --------------------------------------------------------------------------
# Ridge regression workload: X (m x n) FP32, column j scaled by (j+1)^-1
# --------------------------------------------------------------------------

def ridge_X(m: int, n: int, seed: int) -> np.ndarray:
    X = gaussian((m, n), seed, S_X, dtype=np.float32)
    scale = (1.0 / (np.arange(n, dtype=np.float64) + 1.0)).astype(np.float32)
    X *= scale[None, :]
    return X


def ridge_y(m: int, seed: int) -> np.ndarray:
    return gaussian((m,), seed, S_Y)


# --------------------------------------------------------------------------
# Kernel ridge regression workload: Gaussian-mixture points
# --------------------------------------------------------------------------

def gmm_points(n: int, d: int, seed: int, components: int = 10, mean_var: float = 4.0,
               dtype=np.float32) -> np.ndarray:
    """n points in R^d: component drawn uniformly from `components` equal-weight
    components with means ~ N(0, mean_var I) and unit covariance."""
    means = rng(seed, S_MEANS).standard_normal((components, d)) * np.sqrt(mean_var)
    labels = rng(seed, S_LABEL).integers(0, components, size=n)
    noise = gaussian((n, d), seed, S_NOISE)
    return (means[labels] + noise).astype(dtype)


def median_distance(points: np.ndarray, seed: int, sample: int = 4096) -> float:
    """Median of the pairwise Euclidean distances (i < j) over a fixed seeded
    subsample of at most `sample` points.  Used once to set the Gaussian
    kernel bandwidth sigma (the input recipe, not part of the method)."""
    n = points.shape[0]
    if n > sample:
        idx = np.sort(rng(seed, S_SUB).choice(n, size=sample, replace=False))
        P = points[idx].astype(np.float64)
    else:
        P = points.astype(np.float64)
    sq = (P * P).sum(1)
    k = P.shape[0]
    iu = np.triu_indices(k, 1)
    D2 = sq[:, None] + sq[None, :] - 2.0 * (P @ P.T)
    d = np.sqrt(np.maximum(D2[iu], 0.0))
    return float(np.median(d))


def krr_targets(points: np.ndarray, seed: int, noise: float = 0.1) -> np.ndarray:
    """y = sin(w . x) + noise * N(0,1) with w ~ N(0, I)."""
    d = points.shape[1]
    w = rng(seed, S_W).standard_normal(d)
    e = gaussian((points.shape[0],), seed, S_NOISE + 100)
    return np.sin(points.astype(np.float64) @ w) + noise * e


# --------------------------------------------------------------------------
# Small fixtures used by the parity tests
# --------------------------------------------------------------------------

def omega(n: int, ell: int, seed: int) -> np.ndarray:
    """Raw Gaussian test matrix, n x ell, row-major FP64 (before the thin QR)."""
    return gaussian((n, ell), seed, S_OMEGA)


def rhs(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    if nrhs is None:
        return gaussian((n,), seed, S_B)
    return gaussian((nrhs, n), seed, S_B)


def column_indices(n: int, ell: int, seed: int) -> np.ndarray:
    """ell distinct indices of [0, n) (int64), uniformly without replacement."""
    return rng(seed, S_COLS).choice(n, size=ell, replace=False).astype(np.int64)


def selection(n: int, cols: np.ndarray) -> np.ndarray:
    """The n x ell FP64 matrix I[:, cols]."""
    Q = np.zeros((n, len(cols)))
    Q[cols, np.arange(len(cols))] = 1.0
    return Q


def power_starts(n: int, count: int, seed: int) -> np.ndarray:
    """Start vectors g for the randomized power error estimate, [count][n]."""
    return gaussian((count, n), seed, S_G)


def integer_spd(n: int, seed: int, rank: int | None = None, scale: int = 3) -> np.ndarray:
    """Small integer-valued psd matrix G^T G with integer G (rank <= `rank`)."""
    r = n if rank is None else rank
    G = rng(seed, S_X).integers(-scale, scale + 1, size=(r, n)).astype(np.float64)
    return G.T @ G


def integer_vector(n: int, seed: int, scale: int = 5) -> np.ndarray:
    return rng(seed, S_B).integers(-scale, scale + 1, size=n).astype(np.float64)


def integer_omega(n: int, ell: int, seed: int, scale: int = 3) -> np.ndarray:
    return rng(seed, S_OMEGA).integers(-scale, scale + 1, size=(n, ell)).astype(np.float64)


def regularization_path(count: int, lo: float, hi: float) -> np.ndarray:
    return np.logspace(np.log10(lo), np.log10(hi), count)
