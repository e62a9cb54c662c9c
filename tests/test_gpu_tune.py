"""Launch-shape autotuner on the GPU: every slice count it may pick for the
Gaussian kernel-matrix products (one vector and a batch) gives the product to
FP32 accuracy against the FP64 oracle; a solve records its tuned choice and
reuses it; with tuning off nothing is timed or stored."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operators as oops  # noqa: E402

from paper_2110_02820_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ny():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    nyspcg.lib()
    prev = nyspcg.autotune(True)
    yield nyspcg
    nyspcg.autotune(prev)


def T(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def keys_with(ny, prefix, fragment):
    return [k for k in ny.autotune_choices() if k.startswith(prefix) and fragment in k]


@pytest.mark.parametrize("n,d,nvec,prefix", [(5000, 16, 128, "rbf_tc16 passes=3"),
                                              (4100, 9, 70, "rbf_tc16 passes=3"),
                                              (20000, 32, 1, "rbf_gemv")])
def test_every_launch_shape_gives_the_product(ny, n, d, nvec, prefix):
    # one vector: the slice count (1..4); many vectors: vectors per CTA
    # (128, 64, 32) x slices, coded as shape index * 8 + slices
    P = wl.gmm_points(n, d, seed=31)
    sigma = wl.median_distance(P, seed=31)
    V = wl.rhs(n, seed=31, nrhs=nvec)
    op = ny.rbf_operator(T(P), sigma)
    mu = 0.5
    ref = oops.rbf_matmat(P, sigma, V.T).T + mu * V
    ny.autotune_clear()
    y0 = ny.nys_op_matvec(op, mu, T(V), mode=1).cpu().numpy()
    npad = (n + 127) // 128 * 128
    keys = keys_with(ny, prefix, f"npad={npad} d={d}")
    assert len(keys) == 1, ny.autotune_choices()
    many = nvec > 2
    codes = [si * 8 + z for si in range(3) for z in (1, 2, 3, 4)] if many else [1, 2, 3, 4]
    assert ny.autotune_choices()[keys[0]] in codes
    assert relerr(y0, ref) <= 1e-5
    outs = []
    for code in codes:
        ny.autotune_set(keys[0], code)
        y = ny.nys_op_matvec(op, mu, T(V), mode=1).cpu().numpy()
        assert relerr(y, ref) <= 1e-5, code
        outs.append(y)
    # the shapes differ only in how the FP32 sums are grouped (over the
    # points, N(0,1) vectors: the terms cancel), each within the 1e-5 of the
    # oracle above; a dropped or doubled slice or vector block would be off
    # by O(1 / slices)
    for y in outs[1:]:
        assert relerr(y, outs[0]) <= 1e-5
    ny.autotune_clear()


def test_batched_solve_tunes_once_and_reuses_the_choice(ny):
    n, d, ell = 3000, 16, 96
    P = wl.gmm_points(n, d, seed=32)
    sigma = wl.median_distance(P, seed=32)
    mus = list(np.repeat(wl.regularization_path(8, 1e-4 * n, 1e-1 * n), 4))
    B = T(np.tile(wl.rhs(n, seed=32, nrhs=4), (8, 1)))
    op = ny.rbf_operator(T(P), sigma)
    f = ny.nys_sketch(op, ell, omega=T(wl.omega(n, ell, 32)), precision=ny.NYS_PREC_MIXED)
    ny.autotune_clear()
    X1, r1, _ = ny.pcg_solve(op, f, mus, B, tol=1e-8, precision=ny.NYS_PREC_MIXED)
    choices = dict(ny.autotune_choices())
    npad = (n + 127) // 128 * 128
    assert len(keys_with(ny, "rbf_tc16 passes=3", f"npad={npad} d={d} nvec=32")) == 1, choices
    X2, r2, _ = ny.pcg_solve(op, f, mus, B, tol=1e-8, precision=ny.NYS_PREC_MIXED)
    assert ny.autotune_choices() == choices
    assert torch.equal(X1, X2)
    assert all(r.status == ny.NYS_OK for r in r1)
    K = oops.rbf_block(P, P, sigma)
    Xg = X1.cpu().numpy()
    Bn = B.cpu().numpy()
    for s in (0, 17, 31):
        xs = np.linalg.solve(K + mus[s] * np.eye(n), Bn[s])
        assert relerr(Xg[s], xs) <= 1e-5
    ny.autotune_clear()


def test_tuning_off_times_nothing(ny):
    n, d = 5000, 16
    P = wl.gmm_points(n, d, seed=33)
    op = ny.rbf_operator(T(P), wl.median_distance(P, seed=33))
    V = T(wl.rhs(n, seed=33, nrhs=64))
    ny.autotune_clear()
    ny.autotune(False)
    try:
        y = ny.nys_op_matvec(op, 0.1, V, mode=1)
        assert ny.autotune_choices() == {}
        assert torch.isfinite(y).all()
    finally:
        ny.autotune(True)


def test_tf32_kernel_selected_by_environment_gives_the_product(tmp_path):
    # NYS_RBF_TF32=1 (read once per process) selects the 3xTF32 kernel for many
    # vectors instead of the FP16-split one: same product to FP32 accuracy
    import json
    import os
    import subprocess
    import sys
    import textwrap
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent("""
        import json, numpy as np, torch
        from oracle import operators as oops
        from paper_2110_02820_gb300 import build, nyspcg as ny, workloads as wl
        build.build()
        P = wl.gmm_points(3000, 16, seed=41)
        sigma = wl.median_distance(P, seed=41)
        V = wl.rhs(3000, seed=41, nrhs=70)
        op = ny.rbf_operator(torch.tensor(P, device="cuda"), sigma)
        y = ny.nys_op_matvec(op, 0.5, torch.tensor(V, device="cuda"), mode=1).cpu().numpy()
        ref = oops.rbf_matmat(P, sigma, V.T).T + 0.5 * V
        keys = [k for k in ny.autotune_choices() if k.startswith("rbf_tc")]
        print(json.dumps([float(np.linalg.norm(y - ref) / np.linalg.norm(ref)), keys]))
    """)
    env = dict(os.environ, NYS_RBF_TF32="1", NYS_TUNE_CACHE=str(tmp_path / "t.json"))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    err, keys = json.loads(out.stdout.strip().splitlines()[-1])
    assert err <= 1e-5
    # the 3xTF32 kernel names its tuner keys by its fixed 64 vectors per CTA
    assert keys and all(k.startswith("rbf_tc S=64") for k in keys), keys
