"""Pins of the oracle's Philox4x32-10 + Box-Muller generator (Algorithm 1,
step 1: Omega with i.i.d. N(0, 1) entries)."""

import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def _hex(ws):
    return [int(w, 16) for w in ws]


def test_known_answer_vectors():
    items = json.load(open(GOLDEN))["items"]
    ctr = np.array([_hex(it["ctr"]) for it in items], dtype=np.uint32)
    key = np.array([_hex(it["key"]) for it in items], dtype=np.uint32)
    out = ph.philox4x32_10(ctr, key)
    for it, row in zip(items, out):
        assert [int(v) for v in row] == _hex(it["expected"]), it["cite"]


def test_counter_and_key_each_change_every_word():
    # a bijection of the counter under a fixed key; flipping one input bit
    # changes all four output words (ten rounds diffuse every bit)
    base = ph.philox4x32_10([[1, 2, 3, 4]], [[5, 6]])[0]
    for j in range(4):
        c = [1, 2, 3, 4]
        c[j] ^= 1
        assert np.all(ph.philox4x32_10([c], [[5, 6]])[0] != base)
    assert np.all(ph.philox4x32_10([[1, 2, 3, 4]], [[5 ^ 1, 6]])[0] != base)


@pytest.mark.parametrize("first,count", [(0, 1), (0, 7), (3, 9), (4, 4), (1001, 333),
                                         (4 * (1 << 32) - 6, 13)])
def test_stream_slices_agree(first, count):
    # any window of the stream equals the same window of a longer draw; the
    # last case crosses from block 2^32 - 2 into block 2^32 (the counter's
    # second word takes the high bits of the block index)
    seed, sid = 0x0123456789ABCDEF, ph.STREAM_OMEGA
    lo = max(first - 5, 0)
    longer = ph.stream_words(seed, sid, lo, count + 12)
    assert np.array_equal(ph.stream_words(seed, sid, first, count),
                          longer[first - lo:first - lo + count])
    g = np.array([(first + t) // 4 for t in range(count)], dtype=np.int64)
    ctr, key = ph.stream_counters(seed, sid, g)
    assert np.all(ctr[:, 0] == g % (1 << 32))
    assert np.all(ctr[:, 1] == ((g >> 32) ^ (sid & 0xFFFFFFFF)))
    assert np.all(key[:, 0] == seed & 0xFFFFFFFF) and np.all(key[:, 1] == seed >> 32)


def test_streams_and_seeds_are_distinct():
    a = ph.stream_words(1, ph.STREAM_OMEGA, 0, 64)
    assert not np.array_equal(a, ph.stream_words(2, ph.STREAM_OMEGA, 0, 64))
    assert not np.array_equal(a, ph.stream_words(1, ph.STREAM_ESTIMATE_BASE, 0, 64))


def test_open_uniform_endpoints_and_exactness():
    w = np.array([0, 1, 511, 512, 0xFFFFFFFF], dtype=np.uint32)
    u = ph.open_uniform(w)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24 and u[2] == 2.0 ** -24
    assert u[3] == 3 * 2.0 ** -24
    assert u[4] == 1.0 - 2.0 ** -24
    assert np.all((u > 0) & (u < 1))
    # exactly representable in single precision: the GPU forms the same numbers
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)


def test_box_muller_closed_forms():
    u1 = np.array([math.exp(-0.5)] * 4)
    u2 = np.array([0.0, 0.25, 0.5, 0.125])
    c, s = ph.box_muller(u1, u2)
    np.testing.assert_allclose(c, [1.0, 0.0, -1.0, math.sqrt(0.5)], atol=1e-15)
    np.testing.assert_allclose(s, [0.0, 1.0, 0.0, math.sqrt(0.5)], atol=1e-15)
    # radius: u1 = e^{-2} gives sqrt(4) = 2 on both branches
    c, s = ph.box_muller(np.array([math.exp(-2.0)]), np.array([0.3]))
    assert abs(math.hypot(c[0], s[0]) - 2.0) < 1e-14


def test_stream_gaussian_is_standard_normal():
    N = 1 << 18
    z = ph.stream_gaussian(7, ph.STREAM_OMEGA, 0, N)
    assert abs(z.mean()) < 5 / math.sqrt(N)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * math.sqrt(24.0 / N)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two branches of a pair, and neighbouring pairs, are uncorrelated
    zz = z.reshape(-1, 4)
    for a, b in [(0, 1), (2, 3), (1, 2), (0, 2)]:
        assert abs(np.corrcoef(zz[:, a], zz[:, b])[0, 1]) < 5 / math.sqrt(len(zz))
    # even elements are the cosine branch of their pair
    w = ph.stream_words(7, ph.STREAM_OMEGA, 0, 4)
    u = ph.open_uniform(w)
    assert z[0] == math.sqrt(-2 * math.log(u[0])) * math.cos(2 * math.pi * u[1])
    assert z[3] == math.sqrt(-2 * math.log(u[2])) * math.sin(2 * math.pi * u[3])


def test_omega_layout():
    n, ell = 37, 5
    Om = ph.omega(n, ell, 3)
    assert Om.shape == (n, ell)
    assert np.array_equal(Om.reshape(-1), ph.stream_gaussian(3, ph.STREAM_OMEGA, 0, n * ell))
