"""Pins of the regularization-path oracle (warm starts, factor reuse; the
procedure of the paper's path experiments, Sec. 6.2): every solution is the
direct solution, the reuse rule holds on the recorded estimates, rebuilt
sketches start at twice the old size, warm starts save iterations, and the
results do not depend on the order the shifts are given in."""

import math

import numpy as np

from oracle import path, pcg
from oracle import nystrom as ny
from paper_2110_02820_gb300 import workloads as wl


def _setup(n=300, seed=1):
    A, _ = wl.dense_spd(n, seed=seed)
    b = wl.rhs(n, seed=seed)
    return A, b


def _draws(n, ell0, ell_max, seed):
    kmax = int(math.ceil(math.log2(ell_max / ell0))) + 1
    return lambda r: (wl.omega(n, ell_max, seed=100 * seed + r),
                      wl.power_starts(n, kmax, seed=100 * seed + r))


MUS = [10.0 ** e for e in range(0, -7, -1)]


def test_solutions_are_direct_solutions_and_reuse_rule_holds():
    n, ell0, ell_max = 300, 8, 128
    A, b = _setup(n)
    out, builds = path.regularization_path(lambda V: A @ V, n, MUS, b, ell0, ell_max, 30.0, 5,
                                           1e-10, 500, _draws(n, ell0, ell_max, 1))
    prev = None
    for mu, o in zip(MUS, out):
        assert o["status"] == pcg.CONVERGED
        xs = np.linalg.solve(A + mu * np.eye(n), b)
        assert np.linalg.norm(o["x"] - xs) <= 1e-8 * np.linalg.norm(xs)
        if prev is None:
            assert o["resketched"] and o["ell"] >= ell0
        else:
            capped = prev["ell"] >= ell_max
            need = not capped and not (prev["E"] <= 30.0 * mu)
            assert o["resketched"] == need
            if need:
                assert o["ell"] >= min(2 * prev["ell"], ell_max)
            else:
                assert o["ell"] == prev["ell"] and np.array_equal(o["U"], prev["U"])
        if o["resketched"] and o["ell"] < ell_max:
            assert o["E"] <= 30.0 * mu          # Algorithm 5 stopped on its rule
        prev = o
    assert 1 < builds < len(MUS)                # reuse happens, and so do rebuilds


def test_extreme_tolerances():
    n, ell0, ell_max = 200, 4, 64
    A, b = _setup(n, seed=2)
    mus = [1e-1, 1e-2, 1e-3]
    _, one = path.regularization_path(lambda V: A @ V, n, mus, b, ell0, ell_max, 1e12, 5, 1e-8,
                                      500, _draws(n, ell0, ell_max, 2))
    assert one == 1                             # the first factor is always good enough
    out, capped = path.regularization_path(lambda V: A @ V, n, mus, b, ell0, ell_max, 1e-12, 5,
                                           1e-8, 500, _draws(n, ell0, ell_max, 2))
    assert capped == 1 and all(o["ell"] == ell_max for o in out)   # first build hits ell_max


def test_warm_start_saves_iterations_and_order_does_not_matter():
    n, ell0, ell_max = 300, 8, 128
    A, b = _setup(n, seed=3)
    out, _ = path.regularization_path(lambda V: A @ V, n, MUS, b, ell0, ell_max, 30.0, 5, 1e-10,
                                      500, _draws(n, ell0, ell_max, 3))
    cold = [pcg.nys_pcg(lambda v: A @ v, mu, b, None,
                        lambda r, o=o, mu=mu: ny.precond_inverse_apply(o["U"], o["lam"], mu, r),
                        1e-10)["iterations"] for mu, o in zip(MUS, out)]
    warm = [o["iterations"] for o in out]
    assert warm[0] == cold[0]
    assert sum(warm[1:]) < sum(cold[1:])
    perm = [3, 0, 6, 1, 5, 2, 4]
    shuffled, _ = path.regularization_path(lambda V: A @ V, n, [MUS[i] for i in perm], b, ell0,
                                           ell_max, 30.0, 5, 1e-10, 500,
                                           _draws(n, ell0, ell_max, 3))
    for j, i in enumerate(perm):
        assert np.array_equal(shuffled[j]["x"], out[i]["x"])
        assert shuffled[j]["iterations"] == out[i]["iterations"]
