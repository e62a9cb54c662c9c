"""Pins for the oracle's Algorithm 3, batched solves, refinement, Algorithm 5
and the KRR adjoint gradient."""

import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krr
from oracle import nystrom as ny
from oracle import operators as ops
from oracle import pcg
from paper_2110_02820_gb300 import workloads as wl


def spd(n, lam, seed):
    Q = wl.orthogonal(n, seed)
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


def ident(r):
    return r.copy()


# ---------------------------------------------------------------- Algorithm 3

def test_unpreconditioned_iterates_match_scipy_cg():
    # P = I reduces Algorithm 3 to textbook CG; scipy's cg is an independent
    # implementation of the same recurrence.
    n, mu = 120, 1e-2
    A = spd(n, wl.power_spectrum(n, 1.0), 1)
    b = wl.rhs(n, 1)
    for k in [1, 3, 10, 25]:
        ours = pcg.nys_pcg(lambda v: A @ v, mu, b, None, ident, tol=0.0, maxit=k)
        ref, _ = spla.cg(A + mu * np.eye(n), b, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=k)
        assert ours["iterations"] == k
        # rounding differences grow with k (kappa ~ 55); a wrong term is O(1)
        assert np.linalg.norm(ours["x"] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_preconditioned_iterates_match_scipy_pcg():
    n, ell, mu = 150, 12, 1e-3
    A = spd(n, wl.power_spectrum(n, 1.5), 2)
    b = wl.rhs(n, 2)
    f = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 2))
    Pinv = lambda r: ny.precond_inverse_apply(f["U"], f["lam"], mu, r)
    M = spla.LinearOperator((n, n), matvec=Pinv)
    for k in [1, 4, 12]:
        ours = pcg.nys_pcg(lambda v: A @ v, mu, b, None, Pinv, tol=0.0, maxit=k)
        ref, _ = spla.cg(A + mu * np.eye(n), b, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=k, M=M)
        assert np.linalg.norm(ours["x"] - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [2, 5, 8])
def test_terminates_in_at_most_n_steps(n):
    # CG solves an n x n SPD system in at most n steps (exact arithmetic;
    # FP64 with kappa <= 100 here).
    lam = np.linspace(1.0, 100.0, n)
    A = spd(n, lam, n)
    b = wl.rhs(n, n)
    out = pcg.nys_pcg(lambda v: A @ v, 0.0, b, None, ident, tol=1e-10, maxit=50)
    assert out["status"] == pcg.CONVERGED and out["iterations"] <= n


def test_integer_case_iteration_count_is_fixed():
    A = wl.integer_spd(8, seed=0)
    b = wl.integer_vector(8, seed=0)
    out = pcg.nys_pcg(lambda v: A @ v, 1.0, b, None, ident, tol=1e-10, maxit=50)
    assert out["status"] == pcg.CONVERGED
    assert out["iterations"] <= 8
    # the residual drop at the last step is many orders of magnitude, so the
    # count does not sit on the threshold
    assert out["res_hist"][-2] > 1e-6 * np.linalg.norm(b)


def test_exact_recovery_preconditioner_converges_in_two_steps():
    # rank(A) <= ell: P^{-1} A_mu acts as (lam_ell + mu) on range(U) and as mu off it;
    # lam_ell = 0 here, so P^{-1} A_mu = mu I up to rounding and CG stops at once.
    n, r, ell, mu = 100, 8, 12, 1e-2
    rng = np.random.default_rng(0)
    Q = np.linalg.qr(rng.standard_normal((n, r)))[0]
    A = (Q * np.linspace(10, 1, r)) @ Q.T
    f = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 0))
    b = wl.rhs(n, 0)
    out = pcg.nys_pcg(lambda v: A @ v, mu, b, None,
                      lambda r_: ny.precond_inverse_apply(f["U"], f["lam"], mu, r_), 1e-10, 50)
    assert out["iterations"] <= 2


def test_solution_matches_dense_cholesky():
    n, ell, mu = 300, 40, 1e-4
    A = spd(n, wl.power_spectrum(n, 1.5), 3)
    b = wl.rhs(n, 3)
    f = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 3))
    out = pcg.nys_pcg(lambda v: A @ v, mu, b, None,
                      lambda r: ny.precond_inverse_apply(f["U"], f["lam"], mu, r), 1e-13, 500)
    xs = pcg.direct_solve(A, mu, b)
    assert out["status"] == pcg.CONVERGED
    kappa = (1 + mu) / (wl.power_spectrum(n, 1.5)[-1] + mu)
    assert np.linalg.norm(out["x"] - xs) / np.linalg.norm(xs) <= kappa * 1e-13 * 10


def test_cg_error_bound_in_energy_norm():
    # Standard CG bound used in Sec. A.3: ||x_t - x*||_{A_mu} <= 2 ((sqrt k - 1)/(sqrt k + 1))^t ||x*||_{A_mu}.
    n, ell, mu = 200, 15, 1e-3
    A = spd(n, wl.power_spectrum(n, 1.5), 4)
    b = wl.rhs(n, 4)
    f = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 4))
    Pinv = lambda r: ny.precond_inverse_apply(f["U"], f["lam"], mu, r)
    ev = ny.preconditioned_spectrum(A, f["U"], f["lam"], mu)
    kap = ev.max() / ev.min()
    rho = pcg.cg_rate(kap)
    Am = A + mu * np.eye(n)
    xs = np.linalg.solve(Am, b)
    en = lambda e: math.sqrt(e @ Am @ e)
    for t in [1, 5, 10, 20]:
        xt = pcg.nys_pcg(lambda v: A @ v, mu, b, None, Pinv, 0.0, t)["x"]
        assert en(xt - xs) <= 2 * rho ** t * en(xs) * (1 + 1e-8)


def test_maxit_and_breakdown_statuses():
    n = 50
    A = spd(n, wl.power_spectrum(n, 3.0), 5)
    b = wl.rhs(n, 5)
    out = pcg.nys_pcg(lambda v: A @ v, 1e-9, b, None, ident, 1e-14, 3)
    assert out["status"] == pcg.MAXIT and out["iterations"] == 3
    out = pcg.nys_pcg(lambda v: -v, 0.0, b, None, ident, 1e-10, 10)
    assert out["status"] == pcg.BREAKDOWN and out["iterations"] == 0


def test_initial_guess_is_used():
    n, mu = 40, 0.1
    A = spd(n, wl.power_spectrum(n, 1.0), 6)
    b = wl.rhs(n, 6)
    xs = pcg.direct_solve(A, mu, b)
    out = pcg.nys_pcg(lambda v: A @ v, mu, b, xs, ident, 1e-8, 10)
    assert out["iterations"] == 0


# ---------------------------------------------------------------- batched

def test_batched_columns_equal_single_solves():
    n, ell = 120, 10
    A = spd(n, wl.power_spectrum(n, 1.5), 7)
    f = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 7))
    mus = wl.regularization_path(4, 1e-5, 1e-1)
    B = wl.rhs(n, 7, nrhs=4)
    pf = lambda mu: (lambda r: ny.precond_inverse_apply(f["U"], f["lam"], mu, r))
    outs = pcg.batched_pcg(lambda v: A @ v, mus, B, pf, 1e-10)
    for s in range(4):
        one = pcg.nys_pcg(lambda v: A @ v, mus[s], B[s], None, pf(mus[s]), 1e-10)
        assert one["iterations"] == outs[s]["iterations"]
        np.testing.assert_array_equal(one["x"], outs[s]["x"])
        xs = pcg.direct_solve(A, mus[s], B[s])
        assert np.linalg.norm(outs[s]["x"] - xs) / np.linalg.norm(xs) < 1e-5


# ---------------------------------------------------------------- refinement

def test_refinement_reaches_fp64_residual():
    m, n, ell, mu = 3000, 200, 40, 1e-3
    X = wl.ridge_X(m, n, seed=8)
    y = wl.ridge_y(m, 8)
    b = X.astype(np.float64).T @ y
    f = ny.rand_nystrom(lambda V: ops.gram_matmat(X, V), wl.omega(n, ell, 8))
    U32 = f["U"].astype(np.float32)
    out = pcg.refine_solve(lambda v: ops.gram_matmat(X, v),
                           lambda v: ops.gram_matmat(X, v, np.float32),
                           lambda r: ny.precond_inverse_apply_f32(U32, f["lam"], mu, r),
                           mu, b, tol=1e-10, inner_tol=1e-4, maxit=500)
    assert out["status"] == pcg.CONVERGED
    assert out["true_res_hist"][-1] <= 1e-10
    A = X.astype(np.float64).T @ X.astype(np.float64)
    xs = pcg.direct_solve(A, mu, b)
    assert np.linalg.norm(out["x"] - xs) / np.linalg.norm(xs) < 1e-7
    # each outer step contracts the true residual
    h = out["true_res_hist"]
    assert np.all(h[1:] < h[:-1])


# ---------------------------------------------------------------- Algorithm 5

def _adaptive_case(seed=0, n=256):
    A = spd(n, wl.power_spectrum(n, 2.0), seed)
    return A, (lambda V: A @ V)


def test_adaptive_stops_at_ell0_with_loose_tolerance():
    A, mm = _adaptive_case()
    n = A.shape[0]
    out = ny.adaptive_nystrom(mm, n, 8, 64, 1e9, 5, wl.omega(n, 64, 1), wl.power_starts(n, 8, 1))
    assert out["ell"] == 8 and out["doublings"] == 0


def test_adaptive_doubles_to_ell_max_with_zero_tolerance():
    A, mm = _adaptive_case()
    n = A.shape[0]
    out = ny.adaptive_nystrom(mm, n, 8, 100, 0.0, 3, wl.omega(n, 100, 1), wl.power_starts(n, 8, 1))
    assert [h["ell"] for h in out["history"]] == [8, 16, 32, 64, 100]
    assert out["ell"] == 100 and out["U"].shape == (n, 100)


def test_adaptive_recovers_low_rank_matrix():
    n, r = 120, 20
    rng = np.random.default_rng(2)
    Q = np.linalg.qr(rng.standard_normal((n, r)))[0]
    A = (Q * np.linspace(5, 1, r)) @ Q.T
    out = ny.adaptive_nystrom(lambda V: A @ V, n, 4, 64, 1e-8, 5, wl.omega(n, 64, 2),
                              wl.power_starts(n, 8, 2))
    assert out["ell"] >= r
    Ahat = (out["U"] * out["lam"]) @ out["U"].T
    assert np.linalg.norm(Ahat - A, 2) <= 1e-10 * 5


def test_adaptive_ratio_rule():
    A, mm = _adaptive_case(3)
    n = A.shape[0]
    mu = 1e-3
    out = ny.adaptive_nystrom(mm, n, 4, 128, 10.0, 0, wl.omega(n, 128, 3), None, rule="ratio", mu=mu)
    assert out["lam"][-1] / mu <= 10.0
    if out["doublings"] > 0:
        assert out["history"][-2]["lam_ell"] / mu > 10.0


def test_adaptive_doubling_count_thm_5_6():
    # Theorem 5.6 with tau = 44, delta = 1/4: with prob >= 3/4 the number of
    # doublings is <= ceil(log2(ell_tilde / ell0)), ell_tilde = 2 ceil(2 d_eff(delta tau mu / 11)) + 1.
    n, mu, ell0 = 256, 1e-3, 4
    lam = wl.power_spectrum(n, 2.0)
    A = spd(n, lam, 5)
    tau, delta = 44.0, 0.25
    ell_tilde = 2 * math.ceil(2 * ny.effective_dimension(lam, delta * tau * mu / 11)) + 1
    cap = math.ceil(math.log2(ell_tilde / ell0))
    ok = 0
    for s in range(12):
        out = ny.adaptive_nystrom(lambda V: A @ V, n, ell0, n, tau * mu, 5, wl.omega(n, n, 40 + s),
                                  wl.power_starts(n, 10, 40 + s), lambda_rule=True)
        ok += out["doublings"] <= cap
    assert ok >= 0.75 * 12


# ---------------------------------------------------------------- KRR adjoint

def test_krr_gradients_match_central_differences():
    P = wl.gmm_points(150, 4, seed=1, dtype=np.float64)
    V = wl.gmm_points(40, 4, seed=2, dtype=np.float64)
    y = wl.krr_targets(P, 1)
    yv = wl.krr_targets(V, 2)
    sigma, mu = 2.5, 0.3

    def dense_solver(s, m):
        K = ops.rbf_block(P, P, s) + m * np.eye(P.shape[0])
        return lambda r: np.linalg.solve(K, r)

    g = krr.krr_loss_and_grads(P, y, V, yv, sigma, mu, dense_solver(sigma, mu))
    h = 1e-4
    L = lambda s, m, yy: krr.krr_loss(P, yy, V, yv, s, m, dense_solver(s, m))[0]
    fd_s = (L(sigma + h, mu, y) - L(sigma - h, mu, y)) / (2 * h)
    fd_m = (L(sigma, mu + h, y) - L(sigma, mu - h, y)) / (2 * h)
    assert abs(g["dL_dsigma"] - fd_s) <= 1e-5 * abs(fd_s) + 1e-10
    assert abs(g["dL_dmu"] - fd_m) <= 1e-5 * abs(fd_m) + 1e-10
    e = np.zeros_like(y)
    for i in [0, 7, 99]:
        e[:] = 0
        e[i] = h
        fd_b = (L(sigma, mu, y + e) - L(sigma, mu, y - e)) / (2 * h)
        assert abs(g["dL_db"][i] - fd_b) <= 1e-5 * abs(fd_b) + 1e-10


def test_krr_gradients_with_pcg_solve_match_dense():
    P = wl.gmm_points(200, 3, seed=3, dtype=np.float64)
    V = wl.gmm_points(30, 3, seed=4, dtype=np.float64)
    y = wl.krr_targets(P, 3)
    yv = wl.krr_targets(V, 4)
    sigma, mu = 1.7, 0.05
    K = ops.rbf_block(P, P, sigma)
    f = ny.rand_nystrom(lambda W: K @ W, wl.omega(200, 30, 3))
    Pinv = lambda r: ny.precond_inverse_apply(f["U"], f["lam"], mu, r)
    psolve = lambda r: pcg.nys_pcg(lambda v: K @ v, mu, r, None, Pinv, 1e-13, 500)["x"]
    dsolve = lambda r: np.linalg.solve(K + mu * np.eye(200), r)
    a = krr.krr_loss_and_grads(P, y, V, yv, sigma, mu, psolve)
    b = krr.krr_loss_and_grads(P, y, V, yv, sigma, mu, dsolve)
    for k in ["loss", "dL_dmu", "dL_dsigma"]:
        assert abs(a[k] - b[k]) <= 1e-8 * abs(b[k])
