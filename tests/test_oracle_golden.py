"""The oracle's convergence-rate helpers against the constants the paper
prints (tests/golden/convergence_constants.json, each entry cited): the
contraction 0.77 and the 3.8 / 3.9 log(2/eps) iteration counts of the
convergence corollaries for kappa <= 56, and the 3.48 log(2/eps) of the
corollary of Theorem 5.6 at tau = 44.  A rate formula without the square
root, or a mistyped 12 tau / 11, misses them."""

import json
import math
import os

import pytest

from oracle import nystrom as ny
from oracle import pcg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "convergence_constants.json")


def items():
    with open(GOLDEN) as f:
        return json.load(f)["items"]


@pytest.mark.parametrize("it", [i for i in items() if "kappa" in i], ids=lambda i: i["cite"])
def test_cg_rate_matches_printed_corollary(it):
    r = pcg.cg_rate(it["kappa"])
    # the paper prints the rate rounded up to two digits
    assert r <= it["rate_printed"] < r + 0.01
    per_log = 1.0 / math.log(1.0 / r)
    # its iteration count per log(2/eps) is an upper bound, rounded up: from
    # the exact rate (3.72) or from the printed 0.77 (3.83)
    assert per_log <= it["iters_per_log_printed"] < 1.0 / math.log(1.0 / it["rate_printed"]) + 0.1
    for eps in (1e-2, 1e-6, 1e-10):
        t = pcg.iterations_to(r, eps)
        assert 2 * r ** t <= eps < 2 * r ** (t - 1)
        assert t <= math.ceil(it["iters_per_log_printed"] * math.log(2 / eps))


@pytest.mark.parametrize("it", [i for i in items() if "tau" in i], ids=lambda i: i["cite"])
def test_adaptive_rate_matches_printed_corollary(it):
    t0 = ny.adaptive_tau0(it["tau"])
    assert t0 == pytest.approx(0.75, abs=1e-15)  # sqrt(1 + 12 * 44 / 11) = 7 exactly
    assert round(1.0 / math.log(1.0 / t0), 2) == it["iters_per_log_printed"]


def test_adaptive_rate_reduces_to_cg_rate():
    # tau0 is the CG rate of kappa = 1 + 12 tau / 11
    for tau in (1.0, 11.0, 44.0, 300.0):
        assert ny.adaptive_tau0(tau) == pytest.approx(pcg.cg_rate(1 + 12 * tau / 11), rel=1e-14)
