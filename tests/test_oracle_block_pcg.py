"""Pins of the block Nystrom PCG oracle (Sec. 5.2, block variant: O'Leary's
block CG with the orthogonalisation pre-processing of Feng, Owen & Peric) to
facts that do not depend on its own code: optimality over the block Krylov
space (brute force), finite termination, reduction to Algorithm 3 for one
right-hand side, invariance under column permutation, the direct solution."""

import numpy as np
import pytest

from oracle import nystrom as ny
from oracle import pcg
from paper_2110_02820_gb300 import workloads as wl


def _problem(n, ell, seed, mu=1e-2):
    A, _ = wl.dense_spd(n, seed=seed)
    o = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, seed))
    pinv = lambda V: ny.precond_inverse_apply(o["U"], o["lam"], mu, V)
    return A, o, pinv, mu


def test_one_rhs_is_algorithm_3():
    A, o, pinv, mu = _problem(200, 16, 1)
    b = wl.rhs(200, seed=1)
    blk = pcg.block_pcg(lambda V: A @ V, mu, b[None], None, pinv, 1e-10)
    one = pcg.nys_pcg(lambda v: A @ v, mu, b, None, pinv, 1e-10)
    assert blk["iterations"] == one["iterations"]
    assert np.linalg.norm(blk["X"][0] - one["x"]) <= 1e-10 * np.linalg.norm(one["x"])
    assert blk["status"] == [pcg.CONVERGED]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_iterate_minimises_energy_error_over_block_krylov_space(k):
    # column j of X_k minimises ||x - x*_j||_{A_mu} over x0_j + span{M^i Z0, i < k},
    # M = P^{-1}(A + mu I), Z0 = P^{-1} R0 (all columns) -- by brute force
    n, s = 40, 3
    A, o, pinv, mu = _problem(n, 5, 2, mu=0.05)
    Amu = A + mu * np.eye(n)
    B = wl.rhs(n, seed=2, nrhs=s)
    X0 = 0.1 * wl.rhs(n, seed=3, nrhs=s)
    out = pcg.block_pcg(lambda V: A @ V, mu, B, X0, pinv, 0.0, maxit=k)
    assert out["iterations"] == k
    R0 = B.T - Amu @ X0.T
    blocks = [pinv(R0)]
    for _ in range(k - 1):
        blocks.append(pinv(Amu @ blocks[-1]))
    W, _ = np.linalg.qr(np.hstack(blocks))
    C = np.linalg.solve(W.T @ Amu @ W, W.T @ R0)
    Xref = X0.T + W @ C
    np.testing.assert_allclose(out["X"].T, Xref, rtol=0, atol=1e-9 * np.abs(Xref).max())


def test_finite_termination_in_ceil_n_over_s_steps():
    # the block Krylov space gains s dimensions per step: n = 12, s = 3 -> 4 steps
    rng = np.random.default_rng(4)
    Qm, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = Qm @ np.diag(np.linspace(1.0, 20.0, 12)) @ Qm.T
    B = rng.standard_normal((3, 12))
    out = pcg.block_pcg(lambda V: A @ V, 0.0, B, None, lambda V: V.copy(), 1e-10)
    assert out["status"] == [pcg.CONVERGED] * 3
    assert out["iterations"] <= 4
    # a single right-hand side needs up to n = 12
    one = pcg.nys_pcg(lambda v: A @ v, 0.0, B[0], None, lambda v: v.copy(), 1e-10)
    assert one["iterations"] > 4


def test_column_permutation_invariance_and_direct_solution():
    n, s = 300, 4
    A, o, pinv, mu = _problem(n, 24, 5)
    B = wl.rhs(n, seed=5, nrhs=s)
    perm = np.array([2, 0, 3, 1])
    a = pcg.block_pcg(lambda V: A @ V, mu, B, None, pinv, 1e-12)
    b = pcg.block_pcg(lambda V: A @ V, mu, B[perm], None, pinv, 1e-12)
    assert abs(a["iterations"] - b["iterations"]) <= 1
    np.testing.assert_allclose(b["X"], a["X"][perm], rtol=0, atol=1e-9 * np.abs(a["X"]).max())
    Xs = np.linalg.solve(A + mu * np.eye(n), B.T).T
    assert np.linalg.norm(a["X"] - Xs) <= 1e-9 * np.linalg.norm(Xs)


def test_zero_and_duplicate_columns():
    n = 150
    A, o, pinv, mu = _problem(n, 12, 6)
    b = wl.rhs(n, seed=6)
    B = np.stack([b, np.zeros(n), b, 2.0 * wl.rhs(n, seed=7)])
    out = pcg.block_pcg(lambda V: A @ V, mu, B, None, pinv, 1e-10)
    assert out["status"] == [pcg.CONVERGED] * 4
    assert np.all(out["X"][1] == 0.0)
    assert np.linalg.norm(out["X"][0] - out["X"][2]) <= 1e-9 * np.linalg.norm(out["X"][0])
    Xs = np.linalg.solve(A + mu * np.eye(n), B.T).T
    assert np.linalg.norm(out["X"] - Xs) <= 1e-8 * np.linalg.norm(Xs)


def test_block_needs_no_more_steps_than_the_slowest_single_solve():
    # O'Leary: the block method's rate depends on (lambda_s + mu)/(lambda_n + mu)
    n, s = 400, 4
    A, o, pinv, mu = _problem(n, 8, 8, mu=1e-4)
    B = wl.rhs(n, seed=8, nrhs=s)
    blk = pcg.block_pcg(lambda V: A @ V, mu, B, None, pinv, 1e-8)
    singles = [pcg.nys_pcg(lambda v: A @ v, mu, B[j], None, pinv, 1e-8)["iterations"]
               for j in range(s)]
    assert blk["status"] == [pcg.CONVERGED] * s
    assert blk["iterations"] < max(singles)


def test_maxit_status():
    A, o, pinv, mu = _problem(200, 4, 9, mu=1e-6)
    B = wl.rhs(200, seed=9, nrhs=2)
    out = pcg.block_pcg(lambda V: A @ V, mu, B, None, pinv, 1e-14, maxit=3)
    assert out["iterations"] == 3 and out["status"] == [pcg.MAXIT] * 2
    assert out["res_hist"].shape == (4, 2)
