"""Pins for the oracle's Algorithm 1, Eq. (5.3), Algorithm 4, Algorithm 2.

Each pin is something the paper or the mathematics fixes independently of
the oracle's code: closed forms, invariants, library routines, brute force.
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import nystrom as ny
from oracle import operators as ops
from paper_2110_02820_gb300 import workloads as wl


def low_rank_psd(n, r, seed, decay=1.0):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, r))
    Q, _ = np.linalg.qr(G)
    lam = decay ** np.arange(r) * (1.0 + rng.random(r))
    return (Q * lam) @ Q.T


def spd_with_spectrum(n, lam, seed):
    Q = wl.orthogonal(n, seed)
    return 0.5 * ((Q * lam) @ Q.T + ((Q * lam) @ Q.T).T), Q


# ---------------------------------------------------------------- eps

@pytest.mark.parametrize("x", [1.0, 1.5, 2.0, 3.999, 1e-300, 7.3e10, 0.1, 1234.5, 2.0 ** 60])
def test_eps_matches_numpy_spacing(x):
    # MATLAB eps(x) is the spacing of doubles at |x|; numpy.spacing computes the same.
    assert ny.eps_spacing(x) == np.spacing(x)
    assert ny.eps_spacing(-x) == np.spacing(x)


def test_eps_float32_matches_numpy_spacing():
    for x in [1.0, 3.0, 1e-20, 12345.678, 2.0 ** 30]:
        assert ny.eps_spacing(x, 23) == float(np.spacing(np.float32(x)))


# ---------------------------------------------------------------- operators

def test_rbf_operator_matches_cdist_kernel():
    from scipy.spatial.distance import cdist
    P = wl.gmm_points(300, 7, seed=3, dtype=np.float64)
    sigma = 2.3
    K = np.exp(-cdist(P, P, "sqeuclidean") / (2 * sigma ** 2))
    V = np.random.default_rng(0).standard_normal((300, 3))
    np.testing.assert_allclose(ops.rbf_matmat(P, sigma, V, row_chunk=64), K @ V, rtol=1e-12, atol=1e-12)
    Kb = ops.rbf_block(P, P, sigma)
    np.testing.assert_allclose(np.diag(Kb), 1.0, rtol=0, atol=0)
    np.testing.assert_array_equal(Kb, Kb.T)
    assert np.linalg.eigvalsh(Kb).min() > -1e-10


def test_gram_operator_matches_explicit():
    X = wl.ridge_X(500, 40, seed=1)
    v = np.random.default_rng(1).standard_normal(40)
    A = X.astype(np.float64).T @ X.astype(np.float64)
    np.testing.assert_allclose(ops.gram_matmat(X, v), A @ v, rtol=1e-12)


def test_rbf_dsigma_matches_finite_difference():
    P = wl.gmm_points(80, 5, seed=2, dtype=np.float64)
    v = np.random.default_rng(2).standard_normal(80)
    s, h = 3.1, 1e-5
    fd = (ops.rbf_matmat(P, s + h, v) - ops.rbf_matmat(P, s - h, v)) / (2 * h)
    np.testing.assert_allclose(ops.rbf_dsigma_matmat(P, s, v), fd, rtol=1e-7, atol=1e-9)


# ---------------------------------------------------------------- Algorithm 1

def test_thin_qr_orthonormal_and_same_range():
    Om = wl.omega(200, 30, seed=0)
    Q = ny.thin_qr(Om)
    np.testing.assert_allclose(Q.T @ Q, np.eye(30), atol=1e-13)
    # Omega = Q (Q^T Omega)
    np.testing.assert_allclose(Q @ (Q.T @ Om), Om, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_exact_recovery_when_rank_below_ell(seed):
    # Sec. 2.2: if rank(A) <= ell, the Nystrom approximation reproduces A.
    n, r, ell = 120, 10, 16
    A = low_rank_psd(n, r, seed)
    out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, seed))
    Ahat = (out["U"] * out["lam"]) @ out["U"].T
    assert np.linalg.norm(Ahat - A, 2) <= 1e-12 * np.linalg.norm(A, 2) * 100
    assert np.all(out["lam"][r:] <= 1e-12 * out["lam"][0])


def test_shift_is_removed_exactly_when_range_is_captured():
    # If range(A) is inside range(Q) (Q orthonormal), Y_nu = Q (S + nu I) and the
    # core returns eig(S) exactly for ANY nu: pins the shift, its removal and the
    # orientation of B = Y_nu C^{-1}.
    n, ell = 60, 8
    Q = ny.thin_qr(wl.omega(n, ell, 5))
    S = np.diag([5.0, 3.0, 2.0, 1.0, 0.5, 0.25, 0.1, 0.0])
    R = np.linalg.qr(np.random.default_rng(1).standard_normal((ell, ell)))[0]
    Score = R @ S @ R.T
    A = Q @ Score @ Q.T
    for nu in [0.0 + 1e-3, 0.3, 2.0]:
        U, lam, nu_used, esc = ny.shifted_core(Q, A @ Q, nu)
        assert esc == 0 and nu_used == nu
        np.testing.assert_allclose(lam, np.diag(S), atol=1e-12)
        np.testing.assert_allclose((U * lam) @ U.T, A, atol=1e-12)


def test_zero_matrix_gives_zero_eigenvalues_for_any_shift():
    Q = ny.thin_qr(wl.omega(30, 5, 1))
    U, lam, nu, _ = ny.shifted_core(Q, np.zeros((30, 5)), 0.7)
    np.testing.assert_allclose(lam, 0.0, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_loewner_order_and_eigenvalue_interlacing(seed):
    # Lemma 2.1: A_nys <= A in the Loewner order; lam_j(A_nys) <= lam_j(A).
    n, ell = 150, 20
    lam_true = wl.power_spectrum(n, 1.2)
    A, _ = spd_with_spectrum(n, lam_true, seed)
    out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, seed + 10))
    Ahat = (out["U"] * out["lam"]) @ out["U"].T
    assert np.linalg.eigvalsh(A - Ahat).min() >= -1e-12
    assert np.all(out["lam"] <= lam_true[:ell] + 1e-12)
    assert np.all(np.diff(out["lam"]) <= 0) and np.all(out["lam"] >= 0)
    np.testing.assert_allclose(out["U"].T @ out["U"], np.eye(ell), atol=1e-12)


def test_matches_unstable_formula_on_well_conditioned_case():
    # Eq. (2.2): A_nys = Y (Omega^T Y)^+ Y^T (fine when well conditioned).
    n, ell = 40, 6
    A, _ = spd_with_spectrum(n, np.linspace(2.0, 1.0, n), 4)
    Om = wl.omega(n, ell, 4)
    out = ny.rand_nystrom(lambda V: A @ V, Om)
    Ahat = (out["U"] * out["lam"]) @ out["U"].T
    Y = A @ Om
    Aun = Y @ np.linalg.pinv(Om.T @ Y) @ Y.T
    np.testing.assert_allclose(Ahat, Aun, atol=1e-12)


def test_depends_only_on_range_of_omega():
    # Lemma 2.1 item 2.
    n, ell = 80, 10
    A, _ = spd_with_spectrum(n, wl.power_spectrum(n, 2.0), 7)
    Om = wl.omega(n, ell, 7)
    R = np.random.default_rng(3).standard_normal((ell, ell)) + 3 * np.eye(ell)
    a = ny.rand_nystrom(lambda V: A @ V, Om)
    b = ny.rand_nystrom(lambda V: A @ V, Om @ R)
    Ha = (a["U"] * a["lam"]) @ a["U"].T
    Hb = (b["U"] * b["lam"]) @ b["U"].T
    np.testing.assert_allclose(Ha, Hb, atol=1e-12)


def test_nu_is_eps_of_frobenius_norm():
    n, ell = 50, 5
    A, _ = spd_with_spectrum(n, wl.power_spectrum(n), 1)
    out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 1))
    assert out["nu"] == np.spacing(np.linalg.norm(A @ out["Q"], "fro"))


def test_expected_error_bound_prop_2_2():
    # Proposition 2.2 (Eq. (2.3)): E||A - A_nys|| <= min_p [...]; the sample mean
    # over 20 seeds stays below the bound.
    n, ell = 200, 24
    lam = wl.power_spectrum(n, 1.0)
    A, _ = spd_with_spectrum(n, lam, 11)
    errs = []
    for s in range(20):
        out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 100 + s))
        errs.append(np.linalg.norm(A - (out["U"] * out["lam"]) @ out["U"].T, 2))
    bound = min((1 + 2 * (ell - p) / (p - 1)) * lam[ell - p] +
                2 * math.e ** 2 * ell / (p * p - 1) * lam[ell - p:].sum()
                for p in range(2, ell - 1))
    assert np.mean(errs) <= bound


def test_shift_escalation_on_indefinite_core():
    # An indefinite "A" makes Omega^T Y_nu indefinite; the core escalates nu and
    # finally reports not psd.
    n, ell = 30, 4
    A = -np.eye(n)
    with pytest.raises(ny.NotPSDError):
        ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 0))


# ---------------------------------------------------------------- Eq. (5.3)

def _factor(n=100, ell=12, seed=0):
    A, _ = spd_with_spectrum(n, wl.power_spectrum(n, 1.5), seed)
    out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, seed + 1))
    return A, out["U"], out["lam"]


def test_precond_identity_off_range_of_U():
    A, U, lam = _factor()
    v = np.random.default_rng(0).standard_normal(U.shape[0])
    v -= U @ (U.T @ v)
    np.testing.assert_allclose(ny.precond_inverse_apply(U, lam, 1e-3, v), v, atol=1e-13)


def test_precond_scales_eigenvectors():
    A, U, lam = _factor()
    mu = 1e-3
    Z = ny.precond_inverse_apply(U, lam, mu, U)
    np.testing.assert_allclose(Z, U * ((lam[-1] + mu) / (lam + mu))[None, :], atol=1e-13)


def test_precond_times_inverse_is_identity_and_spd():
    A, U, lam = _factor()
    n = U.shape[0]
    for mu in [1e-6, 1e-2, 3.0]:
        Pinv = ny.precond_inverse_apply(U, lam, mu, np.eye(n))
        P = ny.precond_apply(U, lam, mu, np.eye(n))
        np.testing.assert_allclose(P @ Pinv, np.eye(n), atol=1e-10)
        np.testing.assert_allclose(Pinv, Pinv.T, atol=1e-14)
        assert np.linalg.eigvalsh(Pinv).min() > 0


def test_float32_precond_apply_exact_case_equals_fp64():
    # U with entries +-1/2 (columns of a 4 x 4 Hadamard matrix over 2), small
    # integer v and shifts for which every coefficient (lam_ell + mu) / (lam + mu)
    # - 1 is a dyadic number: the float32 emulation is exact and must equal the
    # FP64 Eq. (5.3) bit for bit
    H = 0.5 * np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], float)
    U = H[:, :2]
    lam = np.array([7.0, 3.0])
    mu = 1.0
    v = np.array([3.0, -1.0, 2.0, 5.0])
    z32 = ny.precond_inverse_apply_f32(U.astype(np.float32), lam, mu, v.astype(np.float32))
    z64 = ny.precond_inverse_apply(U, lam, mu, v)
    assert np.array_equal(z32.astype(np.float64), z64)
    # and the closed form: P^{-1} u_1 = (lam_2 + mu)/(lam_1 + mu) u_1 = u_1 / 2
    z = ny.precond_inverse_apply_f32(U.astype(np.float32), lam, mu, U[:, 0].astype(np.float32))
    assert np.array_equal(z.astype(np.float64), 0.5 * U[:, 0])


def test_float32_precond_apply_matches_fp64_to_float32_rounding():
    rs = np.random.default_rng(3)
    n, ell, mu = 300, 12, 1e-2
    U = np.linalg.qr(rs.standard_normal((n, ell)))[0]
    lam = np.sort(rs.uniform(0.1, 10.0, ell))[::-1]
    U32 = U.astype(np.float32)
    v32 = rs.standard_normal(n).astype(np.float32)
    z32 = ny.precond_inverse_apply_f32(U32, lam, mu, v32)
    z64 = ny.precond_inverse_apply(U32.astype(np.float64), lam, mu, v32.astype(np.float64))
    assert np.linalg.norm(z32 - z64) <= 1e-6 * np.linalg.norm(z64)


def test_preconditioned_condition_number_with_exact_eigenpairs():
    # With U, Lam the exact top-ell eigenpairs, P^{-1} A_mu has eigenvalues
    # lam_ell + mu (on range U) and lam_j + mu (j > ell): kappa = (lam_ell+mu)/(lam_n+mu).
    n, ell, mu = 80, 9, 1e-3
    lam_true = wl.power_spectrum(n, 1.5)
    A, Q = spd_with_spectrum(n, lam_true, 2)
    ev = ny.preconditioned_spectrum(A, Q[:, :ell], lam_true[:ell], mu)
    np.testing.assert_allclose(ev.max() / ev.min(), (lam_true[ell - 1] + mu) / (lam_true[-1] + mu),
                               rtol=1e-8)


@pytest.mark.parametrize("seed", range(5))
def test_condition_number_bounds_prop_5_3_every_draw(seed):
    # Proposition 5.3 (Eq. (5.4)), deterministic: holds for every draw.
    n, ell, mu = 256, 20, 1e-3
    lam_true = wl.power_spectrum(n, 1.5)
    A, _ = spd_with_spectrum(n, lam_true, seed)
    out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 50 + seed))
    U, lam = out["U"], out["lam"]
    E = np.linalg.norm(A - (U * lam) @ U.T, 2)
    ev = ny.preconditioned_spectrum(A, U, lam, mu)
    kappa = ev.max() / ev.min()
    lam_n, lh = lam_true[-1], lam[-1]
    lower = max((lh + mu) / (lam_n + mu), 1.0)
    upper = (lh + mu + E) * min(1.0 / mu, (lh + lam_n + 2 * mu) / ((lh + mu) * (lam_n + mu)))
    assert lower * (1 - 1e-8) <= kappa <= upper * (1 + 1e-8)
    # the posterior estimate of Sec. 5.4.1 is the first factor of the upper
    # bound times 1/mu, so it bounds kappa too (and is at least the upper bound)
    est = ny.kappa_estimate(lh, mu, E)
    assert upper * (1 - 1e-12) <= est
    assert kappa <= est * (1 + 1e-8)


def test_expected_condition_number_below_28_thm_5_1():
    # Theorem 5.1: ell = 2 ceil(1.5 d_eff(mu)) + 1 gives E[kappa] < 28.
    n, mu = 300, 1e-2
    lam_true = wl.power_spectrum(n, 2.0)
    A, _ = spd_with_spectrum(n, lam_true, 9)
    deff = ny.effective_dimension(lam_true, mu)
    ell = 2 * math.ceil(1.5 * deff) + 1
    kap = []
    for s in range(20):
        out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 300 + s))
        ev = ny.preconditioned_spectrum(A, out["U"], out["lam"], mu)
        kap.append(ev.max() / ev.min())
    assert np.mean(kap) < 28.0


# ---------------------------------------------------------------- Algorithm 4

def test_power_estimate_is_lower_bound_and_converges():
    n, ell = 200, 15
    A, _ = spd_with_spectrum(n, wl.power_spectrum(n, 1.0), 3)
    out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 3))
    U, lam = out["U"], out["lam"]
    E = A - (U * lam) @ U.T
    true = np.linalg.eigvalsh(E).max()
    g = wl.power_starts(n, 1, 3)[0]
    e5 = ny.power_error_estimate(lambda v: A @ v, U, lam, g, 5)
    assert 0 < e5 <= true * (1 + 1e-12)
    e_many = ny.power_error_estimate(lambda v: A @ v, U, lam, g, 400)
    assert abs(e_many - true) <= 1e-6 * true
    # one step is the Rayleigh quotient of the normalised start
    v0 = g / np.linalg.norm(g)
    assert abs(ny.power_error_estimate(lambda v: A @ v, U, lam, g, 1) - v0 @ E @ v0) <= 1e-12 * true


# ---------------------------------------------------------------- Algorithm 2

def test_sketch_and_solve_woodbury_identity():
    # Eq. (4.1) against the dense inverse of A_nys + mu I.
    A, U, lam = _factor(60, 10, 4)
    mu = 0.05
    b = np.random.default_rng(4).standard_normal(60)
    Ahat = (U * lam) @ U.T
    np.testing.assert_allclose(ny.sketch_and_solve(U, lam, mu, b),
                               np.linalg.solve(Ahat + mu * np.eye(60), b), rtol=1e-10)


def _sketch_solve_case(n, seed):
    # fast spectral decay, so that the Theorem 4.2 bounds sit well below 1/mu
    lam_true = np.exp(-np.arange(n) / 2.0)
    A, _ = spd_with_spectrum(n, lam_true, seed)
    return A, lam_true


def test_sketch_and_solve_inverse_error_theorem_4_2():
    # Eq. (4.2): E||(A + mu I)^-1 - (A_nys + mu I)^-1|| <=
    #   (3 + 4 e^2 sr_p(A) / p) lambda_p / (mu (lambda_p + mu)),  ell = 2p - 1.
    # sr_p is taken with the sum from j = p on (the larger of the paper's two
    # statements of the p-stable rank).  A dropped (I - U U^T) / mu term would
    # leave an error ~ 1 / mu = 10, far above the bound (0.42 at p = 16).
    n, p, mu = 150, 16, 0.1
    ell = 2 * p - 1
    A, lam_true = _sketch_solve_case(n, 61)
    lam_p = lam_true[p - 1]
    sr_p = lam_true[p - 1:].sum() / lam_p
    bound = (3 + 4 * math.e ** 2 * sr_p / p) * lam_p / (mu * (lam_p + mu))
    assert bound < 0.1 / mu
    inv = np.linalg.inv(A + mu * np.eye(n))
    errs = []
    for seed in range(20):
        out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 100 + seed))
        approx = np.column_stack([ny.sketch_and_solve(out["U"], out["lam"], mu, e)
                                  for e in np.eye(n)])
        errs.append(np.linalg.norm(inv - approx, 2))
    assert np.mean(errs) <= bound


def test_sketch_and_solve_solution_error_theorem_4_2():
    # Eq. (4.3): with ell = 2 ceil(1.5 d_eff(eps mu)) + 1 the relative error of
    # the sketch-and-solve solution is at most 26 eps in expectation.  Without
    # the (b - U U^T b) / mu term the error exceeds that bound.
    n, mu, eps = 150, 0.1, 0.02
    A, lam_true = _sketch_solve_case(n, 62)
    ell = 2 * math.ceil(1.5 * ny.effective_dimension(lam_true, eps * mu)) + 1
    assert ell < n
    b = wl.rhs(n, 62)
    xs = np.linalg.solve(A + mu * np.eye(n), b)
    errs, errs_no_tail = [], []
    for seed in range(20):
        out = ny.rand_nystrom(lambda V: A @ V, wl.omega(n, ell, 200 + seed))
        U, lam = out["U"], out["lam"]
        xh = ny.sketch_and_solve(U, lam, mu, b)
        errs.append(np.linalg.norm(xh - xs) / np.linalg.norm(xs))
        head = U @ ((U.T @ b) / (lam + mu))
        errs_no_tail.append(np.linalg.norm(head - xs) / np.linalg.norm(xs))
    assert np.mean(errs) <= 26 * eps
    assert np.mean(errs_no_tail) > 26 * eps


def test_effective_dimension_is_trace_formula():
    n, mu = 50, 0.1
    A, _ = spd_with_spectrum(n, wl.power_spectrum(n), 2)
    tr = np.trace(A @ np.linalg.inv(A + mu * np.eye(n)))
    assert abs(ny.effective_dimension(wl.power_spectrum(n), mu) - tr) < 1e-10


# ---------------------------------------------------------------- column sampling (Sec. 2.2)

def test_column_sampling_equals_column_nystrom_formula():
    # Algorithm 1 with Omega = I[:, S] is the classical column Nystrom
    # approximation C W^{-1} C^T (C = A[:, S], W = A[S, S]) up to the shift nu
    n, ell = 60, 12
    A, _ = wl.dense_spd(n, seed=21)
    S = wl.column_indices(n, ell, seed=21)
    o = ny.rand_nystrom(lambda V: A @ V, wl.selection(n, S))
    C, W = A[:, S], A[np.ix_(S, S)]
    ref = C @ np.linalg.solve(W, C.T)
    got = (o["U"] * o["lam"]) @ o["U"].T
    assert np.linalg.norm(got - ref, 2) <= 1e-9 * np.linalg.norm(ref, 2)


def test_column_sampling_recovers_low_rank_matrix():
    # rank(A) = r and rank(A[:, S]) = r: the approximation is A itself (Sec. 2.2)
    n, r, ell = 50, 5, 9
    rng = np.random.default_rng(3)
    F = rng.standard_normal((n, r))
    A = F @ F.T
    S = wl.column_indices(n, ell, seed=4)
    o = ny.rand_nystrom(lambda V: A @ V, wl.selection(n, S))
    got = (o["U"] * o["lam"]) @ o["U"].T
    assert np.linalg.norm(got - A, 2) <= 1e-9 * np.linalg.norm(A, 2)


def test_column_indices_are_distinct_and_seeded():
    a = wl.column_indices(1000, 200, seed=5)
    assert len(np.unique(a)) == 200 and a.min() >= 0 and a.max() < 1000
    assert np.array_equal(a, wl.column_indices(1000, 200, seed=5))
    assert not np.array_equal(a, wl.column_indices(1000, 200, seed=6))
