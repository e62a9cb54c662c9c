"""The allocation-free ridge matvec (for callers that cannot allocate device
memory during the call) against the regular FP32 matvec entry point.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test.  It builds the library itself, so
it also passes when run alone in a fresh process."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2110_02820_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    return nyspcg


@pytest.mark.parametrize("m,n", [(5003, 4096), (1200, 260)])
def test_noalloc_matvec_matches_regular_entry_point_twice(ny, m, n):
    X = wl.ridge_X(m, n, seed=21)
    x64 = wl.rhs(n, seed=21)
    mu = 1e-3
    op = ny.gram_operator(torch.tensor(X, device="cuda"))
    xd = torch.tensor(x64, device="cuda")
    ref = ny.nys_op_matvec(op, mu, xd, mode=1).cpu().numpy()
    x32 = xd.float()
    for _ in range(2):  # two calls in a row share (and reuse) the scratch array
        y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        ny.nys_gram_matvec_f32_noalloc(op, mu, x32, y)
        got = y.double().cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_noalloc_size_limit(ny):
    # n = 6400 is the widest X whose two-stage shared-memory pipeline fits
    # (2 stages x 4 rows x n floats <= 200 KiB): accepted and equal to the
    # regular entry point.  n = 6404 (still a multiple of 4) is rejected
    # before any device work.  With 152 SMs, 6400 columns give 972800
    # partial floats, inside the 2^20 of the scratch array.
    mu = 1e-3
    X = wl.ridge_X(1000, 6400, seed=22)
    op = ny.gram_operator(torch.tensor(X, device="cuda"))
    xd = torch.tensor(wl.rhs(6400, seed=22), device="cuda")
    ref = ny.nys_op_matvec(op, mu, xd, mode=1).cpu().numpy()
    y = torch.full((6400,), float("nan"), dtype=torch.float32, device="cuda")
    ny.nys_gram_matvec_f32_noalloc(op, mu, xd.float(), y)
    got = y.double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)

    n = 6404
    X = torch.zeros((64, n), dtype=torch.float32, device="cuda")
    op = ny.gram_operator(X)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    y = torch.full((n,), 7.0, dtype=torch.float32, device="cuda")
    with pytest.raises(ny.NysError) as e:
        ny.nys_gram_matvec_f32_noalloc(op, 0.0, x, y)
    assert e.value.status == ny.NYS_ERR_ARG
    assert bool((y == 7.0).all())  # untouched
