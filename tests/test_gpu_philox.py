"""GPU parity of the random test matrix of Algorithm 1, step 1 (Omega with
i.i.d. N(0, 1) entries), drawn by the library's Philox4x32-10 + Box-Muller
generator, against the oracle's independent restatement (``oracle.philox``).

Tolerances: the Philox words are integers and must agree bit for bit (and
with the authors' known-answer vectors).  The Gaussian values are computed
on the GPU in FP32 from the same words (uniforms exact in FP32; logf,
sqrtf, sincospif within a few units of 2^-24): with radius at most
sqrt(2 ln 2^24) < 5.8, their distance from the exact FP64 transform is below
4e-6 (the header's stated bound).
"""

import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import philox as oph  # noqa: E402

from paper_2110_02820_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")
GAUSS_TOL = 4e-6


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    return nyspcg


def _bits(a):
    return torch.tensor(np.asarray(a, dtype=np.uint32).view(np.int32), device="cuda")


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_gpu_philox_known_answer_vectors(ny):
    items = json.load(open(GOLDEN))["items"]
    ctr = np.array([[int(w, 16) for w in it["ctr"]] for it in items], dtype=np.uint32)
    key = np.array([[int(w, 16) for w in it["key"]] for it in items], dtype=np.uint32)
    out = _u32(ny.nys_philox4x32_10(_bits(ctr), _bits(key)))
    for it, row in zip(items, out):
        assert [int(v) for v in row] == [int(w, 16) for w in it["expected"]], it["cite"]


def test_gpu_philox_blocks_bit_exact_on_random_counters(ny):
    rs = np.random.default_rng(5)
    ctr = rs.integers(0, 1 << 32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    key = rs.integers(0, 1 << 32, size=(5000, 2), dtype=np.uint64).astype(np.uint32)
    out = _u32(ny.nys_philox4x32_10(_bits(ctr), _bits(key)))
    assert np.array_equal(out, oph.philox4x32_10(ctr, key))


@pytest.mark.parametrize("seed,sid,first,count", [
    (0, 0, 0, 1), (7, oph.STREAM_OMEGA, 0, 4096 * 64 + 3), (123456789012345, oph.STREAM_OMEGA, 5, 999),
    (2, oph.STREAM_ADAPTIVE_BASE + 1024, 2, 2), (3, oph.STREAM_ESTIMATE_BASE + 1, 17, 1000),
    # the block index crosses 2^32 (the counter's second word takes its high bits)
    (11, oph.STREAM_OMEGA, 4 * (1 << 32) - 10, 21),
    ((1 << 64) - 1, (1 << 64) - 1, (1 << 40) + 1, 77)])
def test_gpu_stream_words_bit_exact(ny, seed, sid, first, count):
    w, g = ny.nys_random_stream(seed, sid, first, count)
    assert np.array_equal(_u32(w), oph.stream_words(seed, sid, first, count))
    ref = oph.stream_gaussian(seed, sid, first, count)
    assert np.max(np.abs(g.cpu().numpy() - ref)) <= GAUSS_TOL


def test_gpu_stream_empty_and_bad_arguments(ny):
    w, g = ny.nys_random_stream(1, 2, 0, 0)
    assert w.numel() == 0 and g.numel() == 0
    with pytest.raises(ny.NysError):
        ny.nys_random_stream(1, 2, -1, 4)


def test_gpu_omega_is_standard_normal(ny):
    # Omega as Algorithm 1 draws it (n x ell row-major): moments, normality and
    # column correlations of the GPU values themselves
    n, ell = 8192, 64
    _, g = ny.nys_random_stream(9, ny.NYS_STREAM_OMEGA, 0, n * ell, words=False)
    z = g.cpu().numpy()
    N = z.size
    assert abs(z.mean()) < 5 / math.sqrt(N)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    from scipy import stats
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * math.sqrt(24.0 / N)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    Om = z.reshape(n, ell)
    C = np.corrcoef(Om, rowvar=False)
    off = np.abs(C[~np.eye(ell, dtype=bool)])
    assert off.max() < 5.5 / math.sqrt(n)
    # and within tolerance of the oracle value by value
    assert np.max(np.abs(z - oph.omega(n, ell, 9).reshape(-1))) <= GAUSS_TOL


def test_sketch_draws_omega_from_its_stream(ny):
    # nys_sketch(seed) equals nys_sketch with Omega passed in from the stream
    n, ell = 700, 24
    A, _ = wl.dense_spd(n, seed=3)
    op = ny.dense_operator(torch.tensor(A, device="cuda"))
    _, g = ny.nys_random_stream(21, ny.NYS_STREAM_OMEGA, 0, n * ell, words=False)
    f1 = ny.nys_sketch(op, ell, seed=21)
    f2 = ny.nys_sketch(op, ell, omega=g.reshape(n, ell))
    assert torch.equal(f1.lam(), f2.lam())
    assert torch.equal(f1.U(), f2.U())
    # and the oracle's Omega gives the same lambda_hat to rounding
    f3 = ny.nys_sketch(op, ell, omega=torch.tensor(oph.omega(n, ell, 21), device="cuda"))
    l1, l3 = f1.lam().cpu().numpy(), f3.lam().cpu().numpy()
    assert np.max(np.abs(l1 - l3)) <= 1e-4 * l1[0]
