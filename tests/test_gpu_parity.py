"""GPU parity: every entry point of the C ABI against the FP64 CPU oracle on
the same seeded inputs.  Sizes span several tiles and a ragged tail.

Tolerances:
* FP64 paths: ``x`` within 1e-8 relative of the oracle's Algorithm 3 iterate
  with the same Omega; lambda_hat within 1e-9 relative to lambda_1.
* Mixed paths: ``x`` within 1e-5 relative of the FP64 solution after
  refinement; FP32 matvecs within 1e-5 relative (norm-wise).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nystrom as onys  # noqa: E402
from oracle import operators as oops  # noqa: E402
from oracle import pcg as opcg  # noqa: E402

from paper_2110_02820_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    return nyspcg


def T(a, dtype=None):
    t = torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t if dtype is None else t.to(dtype)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ---------------------------------------------------------------- matvecs

@pytest.mark.parametrize("n", [1, 33, 300, 2048])
def test_dense_matvec(ny, n):
    A, _ = wl.dense_spd(n, seed=n)
    x = wl.rhs(n, seed=1, nrhs=3)
    op = ny.dense_operator(T(A))
    y = ny.nys_op_matvec(op, 0.25, T(x)).cpu().numpy()
    ref = (A @ x.T).T + 0.25 * x
    assert relerr(y, ref) <= 1e-13


@pytest.mark.parametrize("m,n", [(1000, 260), (3001, 512), (5000, 4096), (777, 9000)])
def test_gram_matvec_accurate_and_fast(ny, m, n):
    X = wl.ridge_X(m, n, seed=2)
    x = wl.rhs(n, seed=2, nrhs=2)
    op = ny.gram_operator(T(X))
    ref = oops.gram_matmat(X, x.T).T + 1e-3 * x
    y64 = ny.nys_op_matvec(op, 1e-3, T(x), mode=0).cpu().numpy()
    assert relerr(y64, ref) <= 1e-12
    y32 = ny.nys_op_matvec(op, 1e-3, T(x), mode=1).cpu().numpy()
    assert relerr(y32, ref) <= 1e-5
    # residual product (double-FP32 on the fused path): FP64-level accuracy
    yres = ny.nys_op_matvec(op, 1e-3, T(x), mode=2).cpu().numpy()
    assert relerr(yres, ref) <= 1e-12


@pytest.mark.parametrize("n,d", [(777, 7), (1500, 32), (300, 64)])
def test_rbf_matvec_accurate_and_fast(ny, n, d):
    P = wl.gmm_points(n, d, seed=3)
    sigma = wl.median_distance(P, seed=3)
    x = wl.rhs(n, seed=3)
    op = ny.rbf_operator(T(P), sigma)
    ref = oops.rbf_matmat(P, sigma, x) + 0.1 * x
    y64 = ny.nys_op_matvec(op, 0.1, T(x), mode=0).cpu().numpy()
    assert relerr(y64, ref) <= 1e-12
    y32 = ny.nys_op_matvec(op, 0.1, T(x), mode=1).cpu().numpy()
    assert relerr(y32, ref) <= 1e-5
    # residual product: double-FP32 distances and exponential, FP64-level accuracy
    yres = ny.nys_op_matvec(op, 0.1, T(x), mode=2).cpu().numpy()
    assert relerr(yres, ref) <= 1e-12
    np.testing.assert_allclose(yres, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n,d", [(2500, 32), (1300, 16), (700, 7), (400, 64)])
def test_rbf_residual_products_entrywise(ny, n, d):
    # double-FP32 entries and sums (Sec. 6.5 residual): every output entry within a
    # few units of 2^-46 of the sum of the magnitudes of its terms
    P = wl.gmm_points(n, d, seed=31)
    sigma = wl.median_distance(P, seed=31)
    X = wl.rhs(n, seed=31, nrhs=2)
    X[1] = np.abs(X[1])  # one vector without cancellation
    op = ny.rbf_operator(T(P), sigma)
    Y = ny.nys_op_matvec(op, 0.1, T(X), mode=2).cpu().numpy()
    ref = oops.rbf_matmat(P, sigma, X.T).T + 0.1 * X
    scale = oops.rbf_matmat(P, sigma, np.abs(X).T).T + 0.1 * np.abs(X)
    for q in range(2):
        err = np.abs(Y[q] - ref[q]) / scale[q]
        assert err.max() <= 4e-14, (q, err.max())


# ---------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("n,ell", [(200, 24), (513, 64), (2048, 64), (100, 1), (64, 64)])
def test_sketch_f64_dense(ny, n, ell):
    A, _ = wl.dense_spd(n, seed=5)
    Om = wl.omega(n, ell, seed=5)
    f = ny.nys_sketch(ny.dense_operator(T(A)), ell, omega=T(Om))
    o = onys.rand_nystrom(lambda V: A @ V, Om)
    lam = f.lam().cpu().numpy()
    U = f.U().cpu().numpy()
    assert np.abs(lam - o["lam"]).max() <= 1e-9 * o["lam"][0]
    np.testing.assert_allclose(U.T @ U, np.eye(ell), atol=1e-11)
    Ah_g = (U * lam) @ U.T
    Ah_o = (o["U"] * o["lam"]) @ o["U"].T
    assert np.linalg.norm(Ah_g - Ah_o, 2) <= 1e-9 * o["lam"][0]
    assert f.nu == o["nu"]


def test_sketch_exact_recovery_on_gpu(ny):
    # rank(A) = 6 < ell = 16: U Lam U^T = A (Sec. 2.2); exercises the shifted CholeskyQR path
    n, r, ell = 300, 6, 16
    rng = np.random.default_rng(0)
    Q = np.linalg.qr(rng.standard_normal((n, r)))[0]
    A = (Q * np.linspace(4, 1, r)) @ Q.T
    f = ny.nys_sketch(ny.dense_operator(T(A)), ell, omega=T(wl.omega(n, ell, 0)))
    U, lam = f.U().cpu().numpy(), f.lam().cpu().numpy()
    assert np.linalg.norm((U * lam) @ U.T - A, 2) <= 1e-10 * 4
    assert np.all(lam[r:] <= 1e-10)


def test_sketch_generated_omega_is_seeded_and_interlaces(ny):
    # the drawn Omega itself is compared with the oracle's generator in
    # test_gpu_philox.py; here: same seed, same factor; another seed, another
    # factor; lambda_hat_j <= lambda_j (Lemma 2.1) for the drawn Omega
    n, ell = 500, 20
    A, _ = wl.dense_spd(n, seed=1)
    op = ny.dense_operator(T(A))
    f1 = ny.nys_sketch(op, ell, seed=7)
    f2 = ny.nys_sketch(op, ell, seed=7)
    f3 = ny.nys_sketch(op, ell, seed=8)
    l1, l2, l3 = (f.lam().cpu().numpy() for f in (f1, f2, f3))
    np.testing.assert_array_equal(l1, l2)
    assert not np.array_equal(l1, l3)
    lam_true = wl.power_spectrum(n)
    assert np.all(l1 <= lam_true[:ell] + 1e-12)


@pytest.mark.parametrize("m,n,ell,tf32", [(4000, 512, 64, True), (20000, 1024, 128, True),
                                          (4001, 512, 64, False)])
def test_sketch_mixed_gram(ny, m, n, ell, tf32):
    # m % 4 == 0: the sketch runs on the TF32 tensor cores (operands truncated
    # to 10 mantissa bits, ~1e-3 relative); otherwise on FP32 SIMT (~1e-6).
    X = wl.ridge_X(m, n, seed=6)
    Om = wl.omega(n, ell, seed=6)
    f = ny.nys_sketch(ny.gram_operator(T(X)), ell, omega=T(Om), precision=ny.NYS_PREC_MIXED)
    o = onys.rand_nystrom(lambda V: oops.gram_matmat(X, V), Om)
    lam = f.lam().cpu().numpy()
    assert f.u_dtype == ny.NYS_F32
    tol = 3e-3 if tf32 else 1e-4
    np.testing.assert_allclose(lam[:8], o["lam"][:8], rtol=tol)
    assert np.abs(lam - o["lam"]).max() <= tol * o["lam"][0]
    U = f.U().cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(U.T @ U, np.eye(ell), atol=1e-5)


@pytest.mark.parametrize("n,d,nvec", [(777, 7, 1), (1000, 32, 20), (300, 16, 130), (50, 3, 2),
                                      (4096, 16, 64)])
def test_rbf_tensor_core_products(ny, n, d, nvec):
    # the tensor-core kernel (3xTF32 inner products and products with the
    # vectors): ragged n, one and several 64-vector chunks
    P = wl.gmm_points(n, d, seed=13)
    sigma = wl.median_distance(P, seed=13)
    X = wl.rhs(n, seed=13, nrhs=nvec)
    op = ny.rbf_operator(T(P), sigma)
    Y = ny.nys_op_matvec(op, 0.25, T(X), mode=1).cpu().numpy()
    ref = oops.rbf_matmat(P, sigma, X.T).T + 0.25 * X
    # FP32 accumulation of n terms: each entry within a few units of 2^-24
    # of the sum of the magnitudes of its terms (the condition of the sum)
    scale = oops.rbf_matmat(P, sigma, np.abs(X).T).T + 0.25 * np.abs(X)
    for q in range(nvec):
        assert np.all(np.abs(Y[q] - ref[q]) <= 4e-6 * scale[q]), q
        assert relerr(Y[q], ref[q]) <= 3e-5, q


@pytest.mark.parametrize("n,d,ell", [(700, 5, 40), (3000, 16, 200)])
def test_sketch_rbf_mixed_tensor_cores(ny, n, d, ell):
    # K Omega on the tensor cores with TF32 kernel entries and TF32 Omega
    P = wl.gmm_points(n, d, seed=19)
    sigma = wl.median_distance(P, seed=19)
    Om = wl.omega(n, ell, seed=19)
    f = ny.nys_sketch(ny.rbf_operator(T(P), sigma), ell, omega=T(Om), precision=ny.NYS_PREC_MIXED)
    o = onys.rand_nystrom(lambda V: oops.rbf_matmat(P, sigma, V), Om)
    lam = f.lam().cpu().numpy()
    np.testing.assert_allclose(lam[:8], o["lam"][:8], rtol=3e-3)
    assert np.abs(lam - o["lam"]).max() <= 3e-3 * o["lam"][0]
    U = f.U().cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(U.T @ U, np.eye(ell), atol=1e-5)
    assert f.stats()["shift_escalations"] == 0


def test_sketch_rbf_f64(ny):
    n, d, ell = 700, 5, 40
    P = wl.gmm_points(n, d, seed=9)
    sigma = wl.median_distance(P, seed=9)
    Om = wl.omega(n, ell, seed=9)
    f = ny.nys_sketch(ny.rbf_operator(T(P), sigma), ell, omega=T(Om))
    o = onys.rand_nystrom(lambda V: oops.rbf_matmat(P, sigma, V), Om)
    assert np.abs(f.lam().cpu().numpy() - o["lam"]).max() <= 1e-9 * o["lam"][0]


# ---------------------------------------------------------------- Eq. (5.3)

def test_precond_apply_f64_and_f32(ny):
    n, ell = 1000, 48
    A, _ = wl.dense_spd(n, seed=4)
    Om = wl.omega(n, ell, seed=4)
    f = ny.nys_sketch(ny.dense_operator(T(A)), ell, omega=T(Om))
    U, lam = f.U().cpu().numpy(), f.lam().cpu().numpy()
    V = wl.rhs(n, seed=4, nrhs=3)
    mus = [1e-4, 1e-2, 1.0]
    Z = ny.nys_precond_apply(f, mus, T(V)).cpu().numpy()
    for s in range(3):
        ref = onys.precond_inverse_apply(U, lam, mus[s], V[s])
        assert relerr(Z[s], ref) <= 1e-13
    Z32 = ny.nys_precond_apply(f, mus, T(V, torch.float32)).cpu().numpy()
    for s in range(3):
        ref = onys.precond_inverse_apply(U, lam, mus[s], V[s])
        assert relerr(Z32[s], ref) <= 1e-5


# ---------------------------------------------------------------- Algorithm 3

def _oracle_pcg_dense(A, Om, mu, b, tol):
    o = onys.rand_nystrom(lambda V: A @ V, Om)
    return opcg.nys_pcg(lambda v: A @ v, mu, b, None,
                        lambda r: onys.precond_inverse_apply(o["U"], o["lam"], mu, r), tol, 500)


def test_pcg_dense_config_n2048(ny):
    # dense FP64 workload: n = 2048, lambda_i = (i+1)^-1.5, mu = 1e-4, ell = 64, tol 1e-10
    n, ell, mu, tol = 2048, 64, 1e-4, 1e-10
    A, _ = wl.dense_spd(n, seed=0)
    Om = wl.omega(n, ell, seed=0)
    b = wl.rhs(n, seed=0)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(Om))
    x, res, hist = ny.pcg_solve(op, f, mu, T(b), tol=tol, history=True)
    ref = _oracle_pcg_dense(A, Om, mu, b, tol)
    assert res[0].status == ny.NYS_OK
    assert abs(res[0].iterations - ref["iterations"]) <= 1
    assert relerr(x.cpu().numpy(), ref["x"]) <= 1e-8
    xs = opcg.direct_solve(A, mu, b)
    assert relerr(x.cpu().numpy(), xs) <= 1e-6
    # recurrence residuals: the two factors differ by ~1e-9 lambda_1 (CholeskyQR2 +
    # Jacobi vs Householder + LAPACK), which moves the Krylov path by ~1e-6 ||r_0||
    # in mid-iteration; a wrong alpha or beta would be O(||r_0||)
    h = hist[0].cpu().numpy()
    k = min(len(ref["res_hist"]), res[0].iterations + 1)
    assert np.abs(h[:k] - ref["res_hist"][:k]).max() <= 1e-5 * ref["res_hist"][0]
    np.testing.assert_allclose(h[:10], ref["res_hist"][:10], rtol=1e-9)


def test_pcg_integer_case_iteration_count_identical(ny):
    A = wl.integer_spd(8, seed=0)
    b = wl.integer_vector(8, seed=0)
    op = ny.dense_operator(T(A))
    x, res, _ = ny.pcg_solve(op, None, 1.0, T(b), tol=1e-10)
    ref = opcg.nys_pcg(lambda v: A @ v, 1.0, b, None, lambda r: r.copy(), 1e-10, 50)
    assert res[0].iterations == ref["iterations"]
    assert relerr(x.cpu().numpy(), ref["x"]) <= 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,ell,rank", [(8, 2, 4), (12, 3, 6), (16, 4, 8), (24, 5, 10)])
def test_pcg_integer_case_nystrom_iteration_counts_identical(ny, seed, n, ell, rank):
    # integer-valued A = G^T G of rank r, integer b and raw Omega: Algorithm
    # 1's factor and Algorithm 3 with the Eq. (5.3) preconditioner give the
    # oracle's iteration count exactly.  range(U) lies in range(A), so
    # P^{-1}(A + mu I) has at most r + 1 distinct eigenvalues and the
    # recurrence terminates within r + 1 steps with a residual drop of many
    # orders at the last one: no step ends near the stopping threshold.
    # (Full-rank integer matrices converge gradually, and there the last
    # step can land within rounding of the threshold.)
    mu = 1.0
    A = wl.integer_spd(n, seed=seed, rank=rank)
    b = wl.integer_vector(n, seed=seed)
    Om = wl.integer_omega(n, ell, seed=seed)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(Om))
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), tol=1e-10)
    o = onys.rand_nystrom(lambda V: A @ V, Om)
    ref = opcg.nys_pcg(lambda v: A @ v, mu, b, None,
                       lambda r: onys.precond_inverse_apply(o["U"], o["lam"], mu, r), 1e-10, 50)
    assert res[0].status == ny.NYS_OK and ref["status"] == opcg.CONVERGED
    assert res[0].iterations == ref["iterations"], (res[0].iterations, ref["iterations"])
    assert res[0].iterations <= rank + 1
    assert relerr(x.cpu().numpy(), ref["x"]) <= 1e-10
    assert np.abs(f.lam().cpu().numpy() - o["lam"]).max() <= 1e-10 * o["lam"][0]


def test_pcg_plain_cg_and_maxit(ny):
    n = 500
    A, _ = wl.dense_spd(n, seed=3)
    b = wl.rhs(n, seed=3)
    op = ny.dense_operator(T(A))
    x, res, _ = ny.pcg_solve(op, None, 1e-2, T(b), tol=1e-10, maxit=7)
    ref = opcg.nys_pcg(lambda v: A @ v, 1e-2, b, None, lambda r: r.copy(), 1e-10, 7)
    assert res[0].status == ny.NYS_ERR_MAXIT and ref["status"] == opcg.MAXIT
    assert res[0].iterations == 7
    assert relerr(x.cpu().numpy(), ref["x"]) <= 1e-10


def test_pcg_initial_guess(ny):
    n, ell, mu = 400, 30, 1e-3
    A, _ = wl.dense_spd(n, seed=8)
    b = wl.rhs(n, seed=8)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 8)))
    xs = opcg.direct_solve(A, mu, b)
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), x=T(xs), tol=1e-8)
    assert res[0].iterations == 0


def test_pcg_batched_columns_equal_single_solves(ny):
    n, ell = 700, 40
    A, _ = wl.dense_spd(n, seed=11)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 11)))
    mus = list(wl.regularization_path(6, 1e-6, 1e-1))
    B = wl.rhs(n, seed=11, nrhs=6)
    X, res, _ = ny.pcg_solve(op, f, mus, T(B), tol=1e-10)
    for s in range(6):
        x1, r1, _ = ny.pcg_solve(op, f, mus[s], T(B[s]), tol=1e-10)
        # the same recurrence; with >= 4 systems the two passes over U serve a
        # group of systems at once, so the sums round in another order
        assert abs(r1[0].iterations - res[s].iterations) <= 1
        assert relerr(X[s].cpu().numpy(), x1.cpu().numpy()) <= 1e-10 * (1 + 1 / mus[s])
        xs = opcg.direct_solve(A, mus[s], B[s])
        assert relerr(X[s].cpu().numpy(), xs) <= 1e-10 * (1 + 1 / mus[s]) * 10


def test_pcg_mixed_gram_refinement(ny):
    m, n, ell, mu = 20000, 1024, 128, 1e-3
    X = wl.ridge_X(m, n, seed=12)
    y = wl.ridge_y(m, 12)
    X64 = X.astype(np.float64)
    b = X64.T @ y
    op = ny.gram_operator(T(X))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 12)), precision=ny.NYS_PREC_MIXED)
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert res[0].status == ny.NYS_OK
    assert res[0].rel_residual <= 1e-8
    xg = x.cpu().numpy()
    # oracle: true FP64 residual and the direct solution
    r = b - (X64.T @ (X64 @ xg) + mu * xg)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-8
    xs = opcg.direct_solve(X64.T @ X64, mu, b)
    assert relerr(xg, xs) <= 1e-5


def test_mixed_preconditioner_keeps_fp64_iteration_count(ny):
    # lambda_1 / (lambda_ell + mu) ~ 1e6: the mixed factor's U must be
    # orthonormal far below 1e-6 for P^{-1} to stay positive definite and as
    # strong as the FP64 one (Eq. (5.3)); the iteration counts must agree.
    m, n, ell, mu = 20000, 2048, 512, 1e-3
    X = wl.ridge_X(m, n, seed=15)
    b = wl.rhs(n, seed=15)
    op = ny.gram_operator(T(X))
    Om = T(wl.omega(n, ell, 15))
    fm = ny.nys_sketch(op, ell, omega=Om, precision=ny.NYS_PREC_MIXED)
    U = fm.U().double()
    assert (U.T @ U - torch.eye(ell, dtype=torch.float64, device=U.device)).abs().max() <= 2e-6
    f64 = ny.nys_sketch(op, ell, omega=Om)
    _, r64, _ = ny.pcg_solve(op, f64, mu, T(b), tol=1e-8)
    _, rm, _ = ny.pcg_solve(op, fm, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert r64[0].status == ny.NYS_OK and rm[0].status == ny.NYS_OK, (r64, rm)
    assert rm[0].iterations <= 2 * r64[0].iterations + 10, (r64, rm)


@pytest.fixture
def reliable_mode(ny):
    prev = ny.pcg_reliable()
    yield
    ny.pcg_reliable(prev)


@pytest.mark.parametrize("kind", ["gram", "dense"])
def test_reliable_updates_match_refinement_and_fp64(ny, kind, reliable_mode):
    # one system, mixed precision: the FP32 recurrence with reliable updates
    # (residual replacement, iterate in FP64) against the restarted
    # refinement loop and FP64 PCG: same solution to the mixed tolerance, the
    # stated residual, and no more products than refinement
    if kind == "gram":
        m, n, ell, mu = 20000, 2048, 512, 1e-3
        X = wl.ridge_X(m, n, seed=16)
        op = ny.gram_operator(T(X))
        A = X.astype(np.float64).T @ X.astype(np.float64)
    else:
        n, ell, mu = 1500, 40, 1e-4
        A, _ = wl.dense_spd(n, seed=16)
        op = ny.dense_operator(T(A))
    xs = opcg.direct_solve(A, mu, wl.rhs(n, 16))
    b = T(wl.rhs(n, 16))
    Om = T(wl.omega(n, ell, 16))
    fm = ny.nys_sketch(op, ell, omega=Om, precision=ny.NYS_PREC_MIXED)
    ny.pcg_reliable(1)
    x1, r1, _ = ny.pcg_solve(op, fm, mu, b, tol=1e-8, precision=ny.NYS_PREC_MIXED)
    ny.pcg_reliable(0)
    x0, r0, _ = ny.pcg_solve(op, fm, mu, b, tol=1e-8, precision=ny.NYS_PREC_MIXED)
    f64 = ny.nys_sketch(op, ell, omega=Om)
    _, r64, _ = ny.pcg_solve(op, f64, mu, b, tol=1e-8)
    for r in (r1[0], r0[0], r64[0]):
        assert r.status == ny.NYS_OK, (r1, r0, r64)
    assert r1[0].rel_residual <= 1e-8 and r1[0].escalated == 0
    assert relerr(x1.cpu().numpy(), xs) <= 1e-5
    assert relerr(x0.cpu().numpy(), xs) <= 1e-5
    # the recurrence keeps its Krylov space across corrections: no more
    # products than the restarted loop, give or take rounding
    assert r1[0].iterations <= r0[0].iterations + 5, (r1, r0, r64)


def test_reliable_updates_fall_back_to_escalation(ny, reliable_mode):
    # a dense system whose FP32 products carry an error comparable to mu (40
    # eigenvalues in [1e-2, 1], the rest in [1e-10, 3e-9], mu = 1e-7: FP32
    # products err by ~6e-8 ||A||) while the preconditioned system is well
    # conditioned and FP64 residuals resolve 1e-8 (kappa u_64 ~ 1e-9): the
    # reliable recurrence cannot reach the tolerance, hands the system to the
    # escalating loop, whose FP64 inner solves do
    n, ell, mu = 600, 48, 1e-7
    lam = np.concatenate([np.logspace(0, -2, 40), np.logspace(np.log10(3e-9), -10, n - 40)])
    A, _ = wl.dense_spd(n, seed=17, eigenvalues=lam)
    b = wl.rhs(n, seed=17)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 17)), precision=ny.NYS_PREC_MIXED)
    ny.pcg_reliable(1)
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED, maxit=300)
    assert res[0].status == ny.NYS_OK and res[0].rel_residual <= 1e-8, res
    assert res[0].escalated == 1
    xs = opcg.direct_solve(A, mu, b)
    assert relerr(x.cpu().numpy(), xs) <= 1e-5


def test_precond_apply_orthonormalises_fp32_factor(ny):
    # An FP32 U has U^T U = I + E.  The apply uses the orthonormal basis
    # V = U (I + E)^{-1/2} of the same range (to first order in E): compared in
    # FP64 with Eq. (5.3) built on the exactly orthonormalised V, the error is
    # second order in ||E||, while the formula taken with U itself is off by ~||E||.
    m, n, ell, mu = 4000, 1024, 256, 1e-3
    X = wl.ridge_X(m, n, seed=60)
    op = ny.gram_operator(T(X))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 60)), precision=ny.NYS_PREC_MIXED)
    U = f.U().double().cpu().numpy()
    lam = f.lam().cpu().numpy()
    G = U.T @ U
    w, Q = np.linalg.eigh(G)
    V = U @ (Q * w ** -0.5) @ Q.T
    v = wl.rhs(n, seed=60, nrhs=3)
    z = ny.nys_precond_apply(f, mu, T(v)).cpu().numpy()
    ref = onys.precond_inverse_apply(V, lam, mu, v.T).T
    naive = onys.precond_inverse_apply(U, lam, mu, v.T).T
    e_fix, e_naive = relerr(z, ref), relerr(naive, ref)
    assert np.abs(G - np.eye(ell)).max() > 1e-8          # the defect is there
    assert e_fix <= 1e-9, (e_fix, e_naive)
    assert e_naive > 10 * e_fix, (e_fix, e_naive)


def test_mixed_pcg_with_lambda_ratio_below_fp32_orthogonality(ny):
    # (lambda_ell + mu) / lambda_1 ~ 1e-7 sits below the FP32 defect ||U^T U - I||
    # (~ 1e-7 sqrt(ell)); with the orthonormalised apply the mixed solve keeps
    # the FP64 iteration count.
    m, n, ell, mu = 20000, 4096, 1024, 1e-4
    X = wl.ridge_X(m, n, seed=61)
    b = wl.rhs(n, seed=61)
    op = ny.gram_operator(T(X))
    Om = T(wl.omega(n, ell, 61))
    fm = ny.nys_sketch(op, ell, omega=Om, precision=ny.NYS_PREC_MIXED)
    f64 = ny.nys_sketch(op, ell, omega=Om)
    lam = f64.lam().cpu().numpy()
    assert (lam[-1] + mu) / lam[0] < 1e-6
    _, r64, _ = ny.pcg_solve(op, f64, mu, T(b), tol=1e-8)
    _, rm, _ = ny.pcg_solve(op, fm, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert r64[0].status == ny.NYS_OK and rm[0].status == ny.NYS_OK, (r64, rm)
    assert rm[0].iterations <= 2 * r64[0].iterations + 10, (r64, rm)


def test_pcg_f64_gram_matches_oracle(ny):
    m, n, ell, mu = 6000, 300, 40, 1e-2
    X = wl.ridge_X(m, n, seed=13)
    b = wl.rhs(n, seed=13)
    Om = wl.omega(n, ell, 13)
    op = ny.gram_operator(T(X))
    f = ny.nys_sketch(op, ell, omega=T(Om))
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), tol=1e-10)
    mm = lambda V: oops.gram_matmat(X, V)
    o = onys.rand_nystrom(mm, Om)
    ref = opcg.nys_pcg(lambda v: mm(v), mu, b, None,
                       lambda r: onys.precond_inverse_apply(o["U"], o["lam"], mu, r), 1e-10, 500)
    assert abs(res[0].iterations - ref["iterations"]) <= 1
    assert relerr(x.cpu().numpy(), ref["x"]) <= 1e-8


def test_pcg_rbf_mixed_refinement(ny):
    n, d, ell = 3000, 8, 100
    P = wl.gmm_points(n, d, seed=14)
    sigma = wl.median_distance(P, seed=14)
    mu = 1e-6 * n * 100
    b = wl.rhs(n, seed=14)
    op = ny.rbf_operator(T(P), sigma)
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 14)), precision=ny.NYS_PREC_MIXED)
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert res[0].status == ny.NYS_OK, res
    K = oops.rbf_block(P, P, sigma)
    xs = opcg.direct_solve(K, mu, b)
    assert relerr(x.cpu().numpy(), xs) <= 1e-5


@pytest.mark.parametrize("n,ell", [(2000, 400), (3001, 512)])
def test_batched_rbf_regularization_path(ny, n, ell):
    # the regularisation-path recipe over its full range: 8 shifts log-spaced
    # in [1e-8, 1e-1] n times 4 right-hand sides = 32 systems sharing one
    # factor; the batched FP32 kernel matvec serves all of them.  At the
    # smallest shifts the FP32 products' error is comparable to mu, so those
    # systems escalate to FP64-accurate inner solves; every system must reach
    # 1e-8 and match the direct solution.
    d = 16
    P = wl.gmm_points(n, d, seed=41)
    sigma = wl.median_distance(P, seed=41)
    mus = np.repeat(wl.regularization_path(8, 1e-8 * n, 1e-1 * n), 4)
    B = wl.rhs(n, seed=41, nrhs=4)
    B = np.tile(B, (8, 1))
    op = ny.rbf_operator(T(P), sigma)
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 41)), precision=ny.NYS_PREC_MIXED)
    X, res, _ = ny.pcg_solve(op, f, list(mus), T(B), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    K = oops.rbf_block(P, P, sigma)
    Xg = X.cpu().numpy()
    for s in range(len(mus)):
        assert res[s].status == ny.NYS_OK, (s, mus[s], res[s])
        assert res[s].rel_residual <= 1e-8
    for m in range(8):
        xs = opcg.direct_solve(K, mus[4 * m], B[4 * m:4 * m + 4].T).T
        for j in range(4):
            assert relerr(Xg[4 * m + j], xs[j]) <= 1e-5, (m, j)
    # the largest shifts stay on FP32 inner solves, the smallest escalate
    assert not any(r.escalated for r in res[-8:])
    assert all(r.escalated for r in res[:4])
    # systems converge unevenly: larger shifts need fewer iterations
    assert res[31].iterations < res[0].iterations


def test_kernel_ridge_recipe_n5000_matches_oracle(ny):
    # the kernel-ridge workload (Sec. 6.5 recipe: 10-component Gaussian
    # mixture in d = 32, sigma = median pairwise distance, shift 1e-6 n) at a
    # seeded n = 5000 subsample: Strategy 2 (ratio rule lambda_ell / mu <= 40,
    # Sec. 5.4.2) from ell0 = 128 up to 2048 in mixed precision, then PCG with
    # FP64-residual refinement to 1e-8, against the oracle's Algorithm 5 on the
    # same Omega and its direct solve
    n, d, ell0, ell_max = 5000, 32, 128, 2048
    P = wl.gmm_points(n, d, seed=0)
    sigma = wl.median_distance(P, seed=0)
    mu = 1e-6 * n
    b = wl.rhs(n, seed=0)
    Om = wl.omega(n, ell_max, 50)
    op = ny.rbf_operator(T(P), sigma)
    f, info = ny.nys_sketch_adaptive(op, ell0, ell_max, ny.NYS_RULE_RATIO, 40.0, 0, mu,
                                     omega=T(Om), precision=ny.NYS_PREC_MIXED)
    K = oops.rbf_block(P, P, sigma)
    o = onys.adaptive_nystrom(lambda V: K @ V, n, ell0, ell_max, 40.0, 0, Om, None, rule="ratio",
                              mu=mu, mantissa_bits=23)
    assert info.ell == o["ell"] and info.doublings == o["doublings"]
    lam = f.lam().cpu().numpy()
    assert np.abs(lam - o["lam"]).max() <= 1e-5 * o["lam"][0]
    x, res, _ = ny.pcg_solve(op, f, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert res[0].status == ny.NYS_OK and res[0].rel_residual <= 1e-8, res
    xs = opcg.direct_solve(K, mu, b)
    assert relerr(x.cpu().numpy(), xs) <= 1e-5
    # the true residual of the returned x, recomputed in FP64 on the CPU
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - (K @ xg + mu * xg)) <= 1.5e-8 * np.linalg.norm(b)


# ---------------------------------------------------------------- Algorithms 4 and 5

def test_power_error_estimate(ny):
    n, ell, q = 600, 30, 5
    A, _ = wl.dense_spd(n, seed=15)
    Om = wl.omega(n, ell, 15)
    g = wl.power_starts(n, 1, 15)[0]
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(Om))
    est = ny.nys_power_err_est(op, f, T(g), q)
    U, lam = f.U().cpu().numpy(), f.lam().cpu().numpy()
    ref = onys.power_error_estimate(lambda v: A @ v, U, lam, g, q)
    assert abs(est - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("rule", ["err", "ratio"])
def test_adaptive_matches_oracle(ny, rule):
    n, ell0, ell_max, q, mu = 512, 8, 200, 5, 1e-3
    A, _ = wl.dense_spd(n, seed=16, eigenvalues=wl.power_spectrum(n, 2.0))
    Om = wl.omega(n, ell_max, 16)
    G = wl.power_starts(n, 8, 16)
    tol = 30 * mu if rule == "err" else 10.0
    op = ny.dense_operator(T(A))
    f, info = ny.nys_sketch_adaptive(op, ell0, ell_max, ny.NYS_RULE_ERR if rule == "err" else ny.NYS_RULE_RATIO,
                                     tol, q, mu, omega=T(Om), g=T(G))
    o = onys.adaptive_nystrom(lambda V: A @ V, n, ell0, ell_max, tol, q, Om, G, rule=rule, mu=mu)
    assert info.ell == o["ell"]
    assert info.doublings == o["doublings"]
    lam = f.lam().cpu().numpy()
    assert np.abs(lam - o["lam"]).max() <= 1e-9 * o["lam"][0]
    if rule == "err":
        assert abs(info.err_est - o["E"]) <= 1e-8 * abs(o["E"])


def test_adaptive_reaches_ell_max(ny):
    n, ell0, ell_max = 300, 8, 100
    A, _ = wl.dense_spd(n, seed=17)
    Om = wl.omega(n, ell_max, 17)
    G = wl.power_starts(n, 8, 17)
    op = ny.dense_operator(T(A))
    f, info = ny.nys_sketch_adaptive(op, ell0, ell_max, ny.NYS_RULE_ERR, 0.0, 3, 1e-3, omega=T(Om),
                                     g=T(G))
    o = onys.adaptive_nystrom(lambda V: A @ V, n, ell0, ell_max, 0.0, 3, Om, G)
    assert info.ell == ell_max == o["ell"]
    assert np.abs(f.lam().cpu().numpy() - o["lam"]).max() <= 1e-9 * o["lam"][0]


# ---------------------------------------------------------------- failure paths

def test_not_psd_is_reported(ny):
    n, ell = 64, 4
    A = -np.eye(n)
    with pytest.raises(ny.NysError) as e:
        ny.nys_sketch(ny.dense_operator(T(A)), ell, omega=T(wl.omega(n, ell, 0)))
    assert e.value.status == ny.NYS_ERR_NOT_PSD


def test_breakdown_is_reported(ny):
    n = 64
    A = -np.eye(n)
    b = wl.rhs(n, seed=0)
    x, res, _ = ny.pcg_solve(ny.dense_operator(T(A)), None, 0.0, T(b), tol=1e-10)
    assert res[0].status == ny.NYS_ERR_BREAKDOWN and res[0].iterations == 0


# ---------------------------------------------------------------- column sampling (Sec. 2.2)

@pytest.mark.parametrize("n,ell", [(300, 24), (2048, 64)])
def test_column_sketch_dense_f64(ny, n, ell):
    A, _ = wl.dense_spd(n, seed=23)
    S = wl.column_indices(n, ell, seed=23)
    f = ny.nys_sketch_columns(ny.dense_operator(T(A)), ell, cols=T(S))
    o = onys.rand_nystrom(lambda V: A @ V, wl.selection(n, S))
    lam, U = f.lam().cpu().numpy(), f.U().cpu().numpy()
    assert np.abs(lam - o["lam"]).max() <= 1e-9 * o["lam"][0]
    Ah_g = (U * lam) @ U.T
    Ah_o = (o["U"] * o["lam"]) @ o["U"].T
    assert np.linalg.norm(Ah_g - Ah_o, 2) <= 1e-9 * o["lam"][0]


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_column_sketch_rbf(ny, precision):
    n, d, ell = 1500, 8, 80
    P = wl.gmm_points(n, d, seed=24)
    sigma = wl.median_distance(P, seed=24)
    S = wl.column_indices(n, ell, seed=24)
    prec = ny.NYS_PREC_F64 if precision == "f64" else ny.NYS_PREC_MIXED
    f = ny.nys_sketch_columns(ny.rbf_operator(T(P), sigma), ell, cols=T(S), precision=prec)
    o = onys.rand_nystrom(lambda V: oops.rbf_matmat(P, sigma, V), wl.selection(n, S))
    lam = f.lam().cpu().numpy()
    tol = 1e-9 if precision == "f64" else 3e-3
    np.testing.assert_allclose(lam[:8], o["lam"][:8], rtol=tol)
    assert np.abs(lam - o["lam"]).max() <= tol * o["lam"][0]


def test_column_sketch_exact_recovery_and_solve(ny):
    # rank(A) = 6 <= ell sampled columns spanning it: U Lam U^T = A, and PCG with
    # that factor converges in at most a few steps (Sec. 2.2, Alg. 3)
    n, r, ell = 400, 6, 20
    rng = np.random.default_rng(7)
    F = rng.standard_normal((n, r))
    A = F @ F.T
    S = wl.column_indices(n, ell, seed=25)
    f = ny.nys_sketch_columns(ny.dense_operator(T(A)), ell, cols=T(S))
    U, lam = f.U().cpu().numpy(), f.lam().cpu().numpy()
    assert np.linalg.norm((U * lam) @ U.T - A, 2) <= 1e-9 * np.linalg.norm(A, 2)
    b = wl.rhs(n, seed=25)
    x, res, _ = ny.pcg_solve(ny.dense_operator(T(A)), f, 1e-2, T(b), tol=1e-10)
    assert res[0].status == ny.NYS_OK and res[0].iterations <= 4, res


def test_column_sketch_seeded_sampling_and_krr_solve(ny):
    n, d, ell = 3000, 8, 100
    P = wl.gmm_points(n, d, seed=26)
    sigma = wl.median_distance(P, seed=26)
    op = ny.rbf_operator(T(P), sigma)
    f1 = ny.nys_sketch_columns(op, ell, seed=11, precision=ny.NYS_PREC_MIXED)
    f2 = ny.nys_sketch_columns(op, ell, seed=11, precision=ny.NYS_PREC_MIXED)
    f3 = ny.nys_sketch_columns(op, ell, seed=12, precision=ny.NYS_PREC_MIXED)
    l1, l2, l3 = (f.lam().cpu().numpy() for f in (f1, f2, f3))
    np.testing.assert_array_equal(l1, l2)
    assert not np.array_equal(l1, l3)
    mu = 1e-6 * n * 100
    b = wl.rhs(n, seed=26)
    x, res, _ = ny.pcg_solve(op, f1, mu, T(b), tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert res[0].status == ny.NYS_OK, res
    xs = opcg.direct_solve(oops.rbf_block(P, P, sigma), mu, b)
    assert relerr(x.cpu().numpy(), xs) <= 1e-5


# ---------------------------------------------------------------- block PCG (Sec. 5.2)

@pytest.mark.parametrize("n,ell,s", [(300, 16, 1), (1000, 32, 4), (777, 24, 7), (2048, 64, 16)])
def test_block_pcg_f64_matches_oracle(ny, n, ell, s):
    A, _ = wl.dense_spd(n, seed=40)
    Om = wl.omega(n, ell, seed=40)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(Om))
    o = onys.rand_nystrom(lambda V: A @ V, Om)
    mu = 1e-3
    B = wl.rhs(n, seed=41, nrhs=s)
    X, res = ny.nys_block_pcg(op, f, mu, T(B), tol=1e-10)
    ref = opcg.block_pcg(lambda V: A @ V, mu, B, None,
                         lambda V: onys.precond_inverse_apply(o["U"], o["lam"], mu, V), 1e-10)
    assert all(r.status == ny.NYS_OK for r in res), res
    # 16 to 44 block steps here: the counts agree to one step
    assert abs(res[0].iterations - ref["iterations"]) <= 1
    Xg = X.cpu().numpy()
    assert relerr(Xg, ref["X"]) <= 1e-8
    Xs = np.linalg.solve(A + mu * np.eye(n), B.T).T
    for j in range(s):
        assert relerr(Xg[j], Xs[j]) <= 1e-8
        # the last digits of a converged recurrence residual are rounding
        assert res[j].rel_residual <= 1e-10 and ref["rel_res"][j] <= 1e-10


def test_block_pcg_one_rhs_equals_pcg_and_fewer_products_than_singles(ny):
    n, ell, s = 1500, 16, 8
    A, _ = wl.dense_spd(n, seed=42)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, seed=42)))
    mu = 1e-5
    B = wl.rhs(n, seed=42, nrhs=s)
    X1, r1 = ny.nys_block_pcg(op, f, mu, T(B[:1]), tol=1e-10)
    x1, p1, _ = ny.pcg_solve(op, f, mu, T(B[0]), tol=1e-10)
    # ~250 steps at a preconditioned kappa ~ 1e5: orthogonality of the
    # residuals is lost long before convergence, and from then on the step
    # count depends on the rounding of every step (finite-precision CG behaves
    # like exact CG on a larger matrix whose eigenvalue clusters depend on
    # the rounding; Greenbaum 1989): the two recurrences, whose reductions
    # round in different orders, may differ by a few steps
    assert abs(r1[0].iterations - p1[0].iterations) <= max(1, 0.02 * p1[0].iterations)
    assert relerr(X1[0].cpu().numpy(), x1.cpu().numpy()) <= 1e-9
    Xb, rb = ny.nys_block_pcg(op, f, mu, T(B), tol=1e-10)
    xs, ps, _ = ny.pcg_solve(op, f, [mu] * s, T(B), tol=1e-10)
    assert all(r.status == ny.NYS_OK for r in rb)
    assert rb[0].iterations < max(p.iterations for p in ps)
    assert relerr(Xb.cpu().numpy(), xs.cpu().numpy()) <= 1e-8


def test_block_pcg_zero_duplicate_columns_and_x0(ny):
    n, ell = 900, 24
    A, _ = wl.dense_spd(n, seed=43)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, seed=43)))
    mu = 1e-3
    b = wl.rhs(n, seed=43)
    B = np.stack([b, np.zeros(n), b, 3.0 * wl.rhs(n, seed=44)])
    X, res = ny.nys_block_pcg(op, f, mu, T(B), tol=1e-10)
    assert all(r.status == ny.NYS_OK for r in res), res
    Xg = X.cpu().numpy()
    assert np.all(Xg[1] == 0.0)
    Xs = np.linalg.solve(A + mu * np.eye(n), B.T).T
    assert relerr(Xg, Xs) <= 1e-8
    # warm start from the solution: no iterations needed
    X2, r2 = ny.nys_block_pcg(op, f, mu, T(B), X=T(Xs), tol=1e-8)
    assert all(r.status == ny.NYS_OK and r.iterations == 0 for r in r2)
    # maxit
    X3, r3 = ny.nys_block_pcg(op, None, 1e-9, T(B), tol=1e-14, maxit=3)
    assert r3[0].iterations == 3 and r3[0].status == ny.NYS_ERR_MAXIT


@pytest.mark.parametrize("kind", ["gram", "rbf"])
def test_block_pcg_mixed_refinement(ny, kind):
    s = 4
    if kind == "gram":
        m, n, ell = 3000, 512, 64
        X = wl.ridge_X(m, n, seed=45)
        op = ny.gram_operator(T(X))
        mu = 1e-3
        Amat = oops.gram_matmat(X, np.eye(n))
    else:
        n, d, ell = 2500, 8, 128
        P = wl.gmm_points(n, d, seed=45)
        sigma = wl.median_distance(P, seed=45)
        op = ny.rbf_operator(T(P), sigma)
        mu = 1e-6 * n * 100
        Amat = oops.rbf_block(P, P, sigma)
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, seed=45)), precision=ny.NYS_PREC_MIXED)
    B = wl.rhs(n, seed=45, nrhs=s)
    Xb, res = ny.nys_block_pcg(op, f, mu, T(B), tol=1e-10, precision=ny.NYS_PREC_MIXED)
    assert all(r.status == ny.NYS_OK for r in res), res
    Xs = np.linalg.solve(Amat + mu * np.eye(n), B.T).T
    for j in range(s):
        assert res[j].rel_residual <= 1e-10
        assert relerr(Xb[j].cpu().numpy(), Xs[j]) <= 1e-6


# ---------------------------------------------------------------- regularization path (Sec. 6.2)

def test_regularization_path_matches_oracle(ny):
    import math
    from oracle import path as opath
    n, ell0, ell_max = 500, 8, 128
    A, _ = wl.dense_spd(n, seed=50)
    b = wl.rhs(n, seed=50)
    mus = [10.0 ** e for e in (-3, 0, -6, -1, -4, -2, -5)]       # any order
    kmax = int(math.ceil(math.log2(ell_max / ell0))) + 1
    draws = lambda r: (wl.omega(n, ell_max, seed=500 + r), wl.power_starts(n, kmax, seed=500 + r))
    ref, builds = opath.regularization_path(lambda V: A @ V, n, mus, b, ell0, ell_max, 30.0, 5,
                                            1e-10, 500, draws)
    oms = np.stack([draws(r)[0] for r in range(len(mus))])
    gss = np.stack([draws(r)[1] for r in range(len(mus))])
    X, out = ny.nys_reg_path(ny.dense_operator(T(A)), mus, T(b), ell0, ell_max, 30.0, 5,
                             omegas=T(oms), gs=T(gss), tol=1e-10)
    assert sum(o["resketched"] for o in out) == builds > 1
    Xg = X.cpu().numpy()
    for i, (o, r) in enumerate(zip(out, ref)):
        assert o["status"] == ny.NYS_OK
        assert o["resketched"] == r["resketched"] and o["ell"] == r["ell"]
        if not math.isnan(r["E"]):
            assert abs(o["err_est"] - r["E"]) <= 1e-6 * r["E"]
        assert abs(o["iterations"] - r["iterations"]) <= 1
        assert relerr(Xg[i], r["x"]) <= 1e-8


def test_regularization_path_mixed_gaussian(ny):
    n, d, ell0, ell_max = 4000, 8, 32, 512
    P = wl.gmm_points(n, d, seed=51)
    sigma = wl.median_distance(P, seed=51)
    op = ny.rbf_operator(T(P), sigma)
    b = wl.rhs(n, seed=51)
    mus = list(np.geomspace(1e-1, 1e-5, 5) * n)
    X, out = ny.nys_reg_path(op, mus, T(b), ell0, ell_max, 30.0, 5, seed=7, tol=1e-8,
                             precision=ny.NYS_PREC_MIXED)
    K = oops.rbf_block(P, P, sigma)
    for i, mu in enumerate(mus):
        assert out[i]["status"] == ny.NYS_OK, out[i]
        xs = np.linalg.solve(K + mu * np.eye(n), b)
        assert relerr(X[i].cpu().numpy(), xs) <= 1e-6
    assert out[0]["resketched"]


# ---------------------------------------------------------------- Algorithm 2 (sketch-and-solve)

def test_sketch_solve_matches_oracle_and_contrasts_with_pcg(ny):
    n, ell, mu = 1500, 48, 1e-3
    A, _ = wl.dense_spd(n, seed=70)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 70)))
    U, lam = f.U().cpu().numpy(), f.lam().cpu().numpy()
    B = wl.rhs(n, seed=70, nrhs=3)
    X = ny.nys_sketch_solve(f, mu, T(B)).cpu().numpy()
    ref = np.stack([onys.sketch_and_solve(U, lam, mu, B[q]) for q in range(3)])
    assert relerr(X, ref) <= 1e-12
    # x solves the Nystrom system (U Lam U^T + mu I) x = b
    R = (U * lam) @ (U.T @ X.T) + mu * X.T - B.T
    assert np.linalg.norm(R) <= 1e-10 * np.linalg.norm(B)
    # the accuracy contrast of Algorithm 2 against PCG on the true system
    xs = np.linalg.solve(A + mu * np.eye(n), B[0])
    xp, res, _ = ny.pcg_solve(op, f, mu, T(B[0]), tol=1e-10)
    e_ss, e_pcg = relerr(X[0], xs), relerr(xp.cpu().numpy(), xs)
    assert e_ss > 100 * e_pcg, (e_ss, e_pcg)
    # FP32 vectors
    X32 = ny.nys_sketch_solve(f, mu, T(B, torch.float32)).cpu().numpy()
    assert relerr(X32, ref) <= 1e-5
