"""PCG under a CUDA graph: the iteration loop of Algorithm 3 run on the device
(one launch of a graph whose conditional WHILE node repeats one iteration),
or captured as a chunk of four iterations and replayed between host checks,
gives bit-identical results to plain stream launches (the same kernels with
the same arguments in the same order); the replayed chunks launch the same
kernels as plain launches, both graph forms stop at the iteration cap, and
timed products keep their event timing."""

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
    prev, prev_loop = nyspcg.pcg_graphs(), nyspcg.pcg_loop()
    yield nyspcg
    nyspcg.pcg_graphs(prev)
    nyspcg.pcg_loop(prev_loop)


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def both_modes(ny, solve, loop_result=True):
    """Runs `solve` with replayed graph chunks, then plain launches (and
    checks the device-side loop against them); returns the chunked and plain
    results and the kernel launches of each."""
    out = []
    for graphs, loop in ((True, False), (False, False), (True, True)):
        ny.pcg_graphs(graphs)
        ny.pcg_loop(loop)
        torch.cuda.synchronize()
        c0, g0 = ny.kernel_launch_count(), ny.pcg_graph_replays()
        r = solve()
        torch.cuda.synchronize()
        replays = ny.pcg_graph_replays() - g0
        # graph modes really launched graphs; plain mode launched none
        assert (replays > 0) if graphs else (replays == 0)
        out.append((r, ny.kernel_launch_count() - c0))
    ny.pcg_graphs(True)
    ny.pcg_loop(True)
    if loop_result:
        same(out[2][0], out[0][0])  # the device-side loop: same kernels, same results
    return out[:2]


def same(ra, rb):
    (xa, resa, _), (xb, resb, _) = ra, rb
    assert torch.equal(xa, xb)
    assert [r.iterations for r in resa] == [r.iterations for r in resb]
    assert [r.status for r in resa] == [r.status for r in resb]


def test_graph_is_on_by_default_and_switchable(ny):
    ny.pcg_graphs(True)
    assert ny.pcg_graphs() is True
    assert ny.pcg_graphs(False) is True
    assert ny.pcg_graphs() is False
    ny.pcg_graphs(True)


@pytest.mark.parametrize("nsys", [1, 6])
def test_graph_replay_bit_identical_dense_f64(ny, nsys):
    n, ell = 700, 40
    A, _ = wl.dense_spd(n, seed=21)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 21)))
    mus = list(wl.regularization_path(nsys, 1e-5, 1e-1))
    B = T(wl.rhs(n, seed=21, nrhs=nsys))
    (g, lg), (p, lp) = both_modes(ny, lambda: ny.pcg_solve(op, f, mus, B, tol=1e-10))
    same(g, p)
    assert lg == lp
    assert all(r.status == ny.NYS_OK for r in g[1])


def test_graph_replay_overruns_the_cap_safely(ny):
    # maxit = 7 is not a multiple of the four iterations a replay holds
    n = 500
    A, _ = wl.dense_spd(n, seed=3)
    op = ny.dense_operator(T(A))
    b = T(wl.rhs(n, seed=3))
    (g, _), (p, _) = both_modes(ny, lambda: ny.pcg_solve(op, None, 1e-2, b, tol=1e-12, maxit=7,
                                                         history=True))
    same(g, p)
    assert g[1][0].status == ny.NYS_ERR_MAXIT and g[1][0].iterations == 7
    hist = g[2][0].cpu().numpy()
    assert np.isfinite(hist[:8]).all() and len(hist) == 8


def test_graph_replay_bit_identical_mixed_gram(ny):
    m, n, ell, mu = 8000, 512, 64, 1e-3
    X = wl.ridge_X(m, n, seed=22)
    op = ny.gram_operator(T(X))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 22)), precision=ny.NYS_PREC_MIXED)
    b = T(wl.rhs(n, seed=22))
    (g, lg), (p, lp) = both_modes(
        ny, lambda: ny.pcg_solve(op, f, mu, b, tol=1e-8, precision=ny.NYS_PREC_MIXED))
    same(g, p)
    assert lg == lp
    assert g[1][0].status == ny.NYS_OK and g[1][0].rel_residual <= 1e-8


def test_graph_replay_bit_identical_batched_rbf(ny):
    # 16 systems: one tensor-core pass over the kernel matrix per iteration,
    # whose scratch is allocated inside the captured graph
    n, d, ell = 1500, 16, 96
    P = wl.gmm_points(n, d, seed=23)
    sigma = wl.median_distance(P, seed=23)
    mus = list(np.repeat(wl.regularization_path(4, 1e-4 * n, 1e-1 * n), 4))
    B = T(np.tile(wl.rhs(n, seed=23, nrhs=4), (4, 1)))
    op = ny.rbf_operator(T(P), sigma)
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 23)), precision=ny.NYS_PREC_MIXED)
    # the first solve of this size also times the product's launch shapes
    # (autotuner); both modes below then launch the same tuned kernels
    ny.pcg_solve(op, f, mus, B, tol=1e-8, precision=ny.NYS_PREC_MIXED)
    (g, lg), (p, lp) = both_modes(
        ny, lambda: ny.pcg_solve(op, f, mus, B, tol=1e-8, precision=ny.NYS_PREC_MIXED))
    same(g, p)
    assert lg == lp
    assert all(r.status == ny.NYS_OK for r in g[1])


def test_graph_replays_keep_product_timing(ny):
    m, n, ell, mu = 8000, 512, 64, 1e-3
    X = wl.ridge_X(m, n, seed=24)
    op = ny.gram_operator(T(X))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 24)), precision=ny.NYS_PREC_MIXED)
    b = T(wl.rhs(n, seed=24))
    timed = []
    for on in (True, False):
        ny.pcg_graphs(on)
        ny.timing_start(4096)
        ny.pcg_solve(op, f, mu, b, tol=1e-8, precision=ny.NYS_PREC_MIXED)
        torch.cuda.synchronize()
        timed.append(ny.timing_stop())
    ny.pcg_graphs(True)
    (ms_g, cnt_g), (ms_p, cnt_p) = timed
    assert cnt_g == cnt_p > 0
    assert ms_g > 0 and ms_p > 0
    # the same kernels: the mean product time agrees within launch jitter
    assert 0.5 < (ms_g / cnt_g) / (ms_p / cnt_p) < 2.0


def test_device_loop_is_one_launch_per_solve(ny):
    # with the device-side loop, an FP64 solve is one graph launch whatever its
    # iteration count, and a batched mixed solve one launch per inner solve
    n, ell = 900, 30
    A, _ = wl.dense_spd(n, seed=25)
    op = ny.dense_operator(T(A))
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 25)))
    b = T(wl.rhs(n, seed=25))
    ny.pcg_graphs(True)
    ny.pcg_loop(True)
    g0 = ny.pcg_graph_replays()
    x, res, _ = ny.pcg_solve(op, f, 1e-5, b, tol=1e-10)
    assert res[0].status == ny.NYS_OK and res[0].iterations > 16
    assert ny.pcg_graph_replays() - g0 == 1
    # 8 systems of a Gaussian kernel, mixed precision: one launch per refinement step
    m, d, ell2 = 1200, 16, 80
    P = wl.gmm_points(m, d, seed=26)
    sigma = wl.median_distance(P, seed=26)
    opk = ny.rbf_operator(T(P), sigma)
    fk = ny.nys_sketch(opk, ell2, omega=T(wl.omega(m, ell2, 26)), precision=ny.NYS_PREC_MIXED)
    mus = list(np.repeat(wl.regularization_path(2, 1e-3 * m, 1e-1 * m), 4))
    B = T(np.tile(wl.rhs(m, seed=26, nrhs=4), (2, 1)))
    ny.pcg_solve(opk, fk, mus, B, tol=1e-8, precision=ny.NYS_PREC_MIXED)  # tuner warm-up
    g0 = ny.pcg_graph_replays()
    X, resk, _ = ny.pcg_solve(opk, fk, mus, B, tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert all(r.status == ny.NYS_OK for r in resk)
    assert ny.pcg_graph_replays() - g0 == max(r.refinements for r in resk)
