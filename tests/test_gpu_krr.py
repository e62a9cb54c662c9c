"""Differentiable KRR: cross-kernel products and the adjoint gradient
(dL/db, dL/dmu, dL/dsigma) against the FP64 oracle and central differences."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import krr as okrr  # noqa: E402
from oracle import operators as oops  # noqa: E402
from paper_2110_02820_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    return nyspcg


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("nt,n,d", [(300, 700, 7), (129, 1000, 16)])
def test_cross_kernel_products(ny, nt, n, d):
    P = wl.gmm_points(n, d, seed=31)
    Tg = wl.gmm_points(nt, d, seed=32)
    sigma = wl.median_distance(P, seed=31)
    v = wl.rhs(n, seed=31, nrhs=2)
    out0 = ny.nys_rbf_cross_matvec(T(Tg), T(P), sigma, T(v), kind=0).cpu().numpy()
    out1 = ny.nys_rbf_cross_matvec(T(Tg), T(P), sigma, T(v), kind=1).cpu().numpy()
    ref0 = oops.rbf_cross_matmat(Tg, P, sigma, v.T).T
    ref1 = oops.rbf_dsigma_matmat(P, sigma, v.T, targets=Tg).T
    np.testing.assert_allclose(out0, ref0, rtol=1e-11, atol=1e-12 * np.abs(ref0).max())
    np.testing.assert_allclose(out1, ref1, rtol=1e-11, atol=1e-12 * np.abs(ref1).max())


def _problem(n=1200, nv=150, d=4, seed=33):
    P = wl.gmm_points(n, d, seed=seed)
    V = wl.gmm_points(nv, d, seed=seed + 1)
    y = wl.krr_targets(P, seed)
    yv = wl.krr_targets(V, seed + 1)
    sigma = wl.median_distance(P, seed=seed)
    mu = 1e-3 * n
    return P, V, y, yv, sigma, mu


def _gpu_grads(ny, P, V, y, yv, sigma, mu, precision, ell=100, tol=1e-12):
    from paper_2110_02820_gb300 import krr
    yt = T(y).requires_grad_(True)
    sg = torch.tensor(sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    m = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    L = krr.validation_loss(T(P), yt, T(V), T(yv), sg, m, ell, precision=precision, tol=tol)
    L.backward()
    return float(L), yt.grad.cpu().numpy(), float(m.grad), float(sg.grad)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_adjoint_gradients_match_oracle(ny, precision):
    P, V, y, yv, sigma, mu = _problem()
    prec = ny.NYS_PREC_F64 if precision == "f64" else ny.NYS_PREC_MIXED
    L, gy, gmu, gsig = _gpu_grads(ny, P, V, y, yv, sigma, mu, prec)
    K = oops.rbf_block(P, P, sigma) + mu * np.eye(P.shape[0])
    ref = okrr.krr_loss_and_grads(P, y, V, yv, sigma, mu, lambda r: np.linalg.solve(K, r))
    tol = 1e-7 if precision == "f64" else 1e-6
    assert abs(L - ref["loss"]) <= tol * abs(ref["loss"])
    assert abs(gmu - ref["dL_dmu"]) <= 10 * tol * abs(ref["dL_dmu"])
    assert abs(gsig - ref["dL_dsigma"]) <= 10 * tol * abs(ref["dL_dsigma"])
    assert np.linalg.norm(gy - ref["dL_db"]) <= 10 * tol * np.linalg.norm(ref["dL_db"])


def test_adjoint_gradients_match_central_differences(ny):
    from paper_2110_02820_gb300 import krr
    P, V, y, yv, sigma, mu = _problem(n=800, nv=100, d=3, seed=35)
    L, gy, gmu, gsig = _gpu_grads(ny, P, V, y, yv, sigma, mu, ny.NYS_PREC_F64)

    def loss(s, m):
        with torch.no_grad():
            return float(krr.validation_loss(T(P), T(y), T(V), T(yv),
                                             torch.tensor(s, dtype=torch.float64, device="cuda"),
                                             torch.tensor(m, dtype=torch.float64, device="cuda"),
                                             100, precision=ny.NYS_PREC_F64, tol=1e-13))

    h = 1e-4
    fd_s = (loss(sigma * (1 + h), mu) - loss(sigma * (1 - h), mu)) / (2 * h * sigma)
    fd_m = (loss(sigma, mu * (1 + h)) - loss(sigma, mu * (1 - h))) / (2 * h * mu)
    assert abs(gsig - fd_s) <= 1e-5 * abs(fd_s)
    assert abs(gmu - fd_m) <= 1e-5 * abs(fd_m)


def test_adjoint_at_the_differentiable_krr_recipe_n5000(ny):
    # the differentiable-KRR workload (GMM points in d = 16, targets
    # sin(w.x) + 0.1 N(0,1), shift 1e-6 n, ell = 2048, mixed precision) at a
    # seeded n = 5000 training subsample with 500 validation points: the
    # loss, dL/dmu, dL/dsigma and dL/db against the oracle's FP64 gradient
    # (dense solves) at 1e-6, and dL/dmu, dL/dsigma against central
    # differences of the GPU loss with h = 1e-4
    from paper_2110_02820_gb300 import krr
    n, nv, d, ell = 5000, 500, 16, 2048
    P = wl.gmm_points(n, d, seed=0)
    V = wl.gmm_points(nv, d, seed=1)
    y, yv = wl.krr_targets(P, 0), wl.krr_targets(V, 1)
    sigma = wl.median_distance(P, seed=0)
    mu = 1e-6 * n
    # tol 1e-10: the FP64 residual of this shift (kappa ~ 1e6) bottoms out near 1e-11
    L, gy, gmu, gsig = _gpu_grads(ny, P, V, y, yv, sigma, mu, ny.NYS_PREC_MIXED, ell=ell,
                                  tol=1e-10)
    K = oops.rbf_block(P, P, sigma) + mu * np.eye(n)
    import scipy.linalg as sla
    c = sla.cho_factor(K)
    ref = okrr.krr_loss_and_grads(P, y, V, yv, sigma, mu, lambda r: sla.cho_solve(c, r))
    assert abs(L - ref["loss"]) <= 1e-6 * abs(ref["loss"])
    assert abs(gmu - ref["dL_dmu"]) <= 1e-6 * abs(ref["dL_dmu"])
    assert abs(gsig - ref["dL_dsigma"]) <= 1e-6 * abs(ref["dL_dsigma"])
    assert np.linalg.norm(gy - ref["dL_db"]) <= 1e-6 * np.linalg.norm(ref["dL_db"])

    def loss(s, m):
        with torch.no_grad():
            return float(krr.validation_loss(T(P), T(y), T(V), T(yv),
                                             torch.tensor(s, dtype=torch.float64, device="cuda"),
                                             torch.tensor(m, dtype=torch.float64, device="cuda"),
                                             ell, precision=ny.NYS_PREC_MIXED, tol=1e-10))

    h = 1e-4
    fd_s = (loss(sigma * (1 + h), mu) - loss(sigma * (1 - h), mu)) / (2 * h * sigma)
    fd_m = (loss(sigma, mu * (1 + h)) - loss(sigma, mu * (1 - h))) / (2 * h * mu)
    # central differences carry O(h^2) truncation and the solves' error
    # divided by h: both below 1e-5 relative here
    assert abs(gsig - fd_s) <= 1e-5 * abs(fd_s)
    assert abs(gmu - fd_m) <= 1e-5 * abs(fd_m)
