"""The seeded input generators shared by the tests, the bench and the oracle
produce the workloads the benchmark configurations state: shapes, dtypes,
spectra, column scales, mixture structure, seeding, and chunk-independent
streams."""

import numpy as np
import pytest

from paper_2110_02820_gb300 import workloads as wl


def test_streams_are_seeded_and_independent():
    a = wl.rhs(1000, 3)
    np.testing.assert_array_equal(a, wl.rhs(1000, 3))
    assert not np.array_equal(a, wl.rhs(1000, 4))
    # another kind of array from the same seed does not repeat this stream
    assert not np.allclose(a, wl.omega(1000, 1, 3)[:, 0])


def test_large_arrays_do_not_depend_on_threading():
    # chunked fills: the rows of a large draw equal the same rows of a larger draw
    X1 = wl.ridge_X(20000, 16, 5)
    X2 = wl.ridge_X(30000, 16, 5)
    np.testing.assert_array_equal(X1, X2[:20000])


def test_dense_workload_spectrum_and_symmetry():
    # dense FP64 workload: A = Q diag((i+1)^-1.5) Q^T, Q orthogonal
    n = 300
    A, lam = wl.dense_spd(n, 0)
    np.testing.assert_allclose(lam, (np.arange(n) + 1.0) ** -1.5)
    np.testing.assert_array_equal(A, A.T)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A))[::-1], lam, atol=1e-13)
    Q = wl.orthogonal(n, 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-12)


def test_ridge_workload_column_scales():
    # ridge workload: X_ij ~ N(0, 1) / (j + 1), FP32
    m, n = 40000, 64
    X = wl.ridge_X(m, n, 1)
    assert X.dtype == np.float32 and X.shape == (m, n)
    sd = X.astype(np.float64).std(0) * (np.arange(n) + 1.0)
    np.testing.assert_allclose(sd, 1.0, atol=0.02)
    assert abs(X.astype(np.float64).mean()) < 0.01


def test_gaussian_mixture_points():
    # kernel workloads: 10 equal-weight components, means N(0, 4 I), unit covariance
    n, d = 20000, 8
    P = wl.gmm_points(n, d, 2)
    assert P.shape == (n, d) and P.dtype == np.float32
    means = wl.rng(2, wl.S_MEANS).standard_normal((10, d)) * 2.0
    labels = wl.rng(2, wl.S_LABEL).integers(0, 10, size=n)
    resid = P.astype(np.float64) - means[labels]
    np.testing.assert_allclose(resid.std(0), 1.0, atol=0.03)
    counts = np.bincount(labels, minlength=10)
    assert counts.min() > 0.8 * n / 10
    # sigma: the median pairwise distance (of the subsample) is of the order of the
    # spread of the means plus the unit noise: sqrt(2 d (4 + 1)) for distinct components
    s = wl.median_distance(P, 2)
    assert 0.5 * np.sqrt(2 * d) < s < 1.5 * np.sqrt(2 * d * 5)


def test_regularization_path_is_log_spaced():
    mus = wl.regularization_path(32, 1e-8, 1e-1)
    assert len(mus) == 32
    np.testing.assert_allclose([mus[0], mus[-1]], [1e-8, 1e-1])
    r = mus[1:] / mus[:-1]
    np.testing.assert_allclose(r, r[0])


@pytest.mark.parametrize("n,ell", [(50, 7), (1000, 64)])
def test_omega_and_columns(n, ell):
    Om = wl.omega(n, ell, 9)
    assert Om.shape == (n, ell) and Om.dtype == np.float64
    cols = wl.column_indices(n, ell, 9)
    assert len(np.unique(cols)) == ell and cols.min() >= 0 and cols.max() < n
    S = wl.selection(n, cols)
    np.testing.assert_array_equal(S.sum(0), 1.0)
    np.testing.assert_array_equal(np.argmax(S, axis=0), cols)


def test_integer_fixtures_are_integer_valued_and_psd():
    A = wl.integer_spd(8, 0)
    assert np.array_equal(A, np.round(A)) and np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > -1e-9
    v = wl.integer_vector(8, 0)
    assert np.array_equal(v, np.round(v))
