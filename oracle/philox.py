"""Counter-based Gaussian test matrices: Philox4x32-10 and Box-Muller, plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1, step 1 draws the test matrix Omega with i.i.d. N(0, 1) entries.
The library draws it on the GPU from a counter-based generator; this module
restates that generator independently, from its published definitions, so
that the GPU draw can be compared with it:

* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11, Sec. 4.2 and Table 2): a 128-bit counter
  (c0, c1, c2, c3) and a 64-bit key (k0, k1); one round computes the two
  32x32 -> 64-bit products M0 c0 and M1 c2 with M0 = 0xD2511F53,
  M1 = 0xCD9E8D57 and maps the counter to
  (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
  between rounds the key is bumped by the Weyl constants
  (0x9E3779B9, 0xBB67AE85); ten rounds.  Pinned by the authors' published
  known-answer vectors (``tests/golden/philox4x32_10_kat.json``).
* The library's stream layout (the documented interface of
  ``nys_random_stream``): element e of stream (seed, sid) is word e mod 4 of
  the block of counter (g mod 2^32, (g >> 32) ^ (sid mod 2^32), sid >> 32,
  0x6e79) under key (seed mod 2^32, seed >> 32), g = e // 4.
* Open uniforms u = (floor(w / 2^9) + 1/2) 2^-23 in (0, 1): 23 bits of the
  word, exactly representable in single and double precision alike.
* Box-Muller (Box & Muller, Ann. Math. Statist. 29, 1958): from a pair of
  independent uniforms, sqrt(-2 ln u1) cos(2 pi u2) and
  sqrt(-2 ln u1) sin(2 pi u2) are independent N(0, 1).  Element pairs
  (0, 1) and (2, 3) of a block take words (0, 1) and (2, 3): the even element
  is the cosine branch, the odd one the sine branch.

Everything here is FP64 and integer arithmetic on numpy uint64 arrays (each
32 x 32-bit product fits 64 bits).
"""

from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
ROUNDS = 10
STREAM_TAG = 0x6e79

# stream identifiers the library uses for its own draws (the header's
# NYS_STREAM_* constants): Algorithm 1's Omega, the blocks of Algorithm 5
# (plus the sketch size reached before the block), Algorithm 4's start
# vectors (plus the estimate's index)
STREAM_OMEGA = 0x4F6D656761
STREAM_ADAPTIVE_BASE = 0x4164610000
STREAM_ESTIMATE_BASE = 0x4573740000


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` ([count, 4] uint32) under keys
    ``key`` ([count, 2] uint32).  Returns [count, 4] uint32."""
    c = np.array(ctr, dtype=np.uint64).reshape(-1, 4).copy()
    k = np.array(key, dtype=np.uint64).reshape(-1, 2).copy()
    for _ in range(ROUNDS):
        p0 = M0 * c[:, 0]
        p1 = M1 * c[:, 2]
        c = np.stack([((p1 >> np.uint64(32)) ^ c[:, 1] ^ k[:, 0]) & MASK32,
                      p1 & MASK32,
                      ((p0 >> np.uint64(32)) ^ c[:, 3] ^ k[:, 1]) & MASK32,
                      p0 & MASK32], axis=1)
        k = np.stack([(k[:, 0] + W0) & MASK32, (k[:, 1] + W1) & MASK32], axis=1)
    return c.astype(np.uint32)


def stream_counters(seed: int, sid: int, g: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Counters and keys of blocks g (int64 array) of stream (seed, sid)."""
    g = np.asarray(g, dtype=np.uint64)
    ctr = np.stack([g & MASK32,
                    (g >> np.uint64(32)) ^ np.uint64(sid & 0xFFFFFFFF),
                    np.full_like(g, (sid >> 32) & 0xFFFFFFFF),
                    np.full_like(g, STREAM_TAG)], axis=1)
    key = np.tile(np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64),
                  (len(g), 1))
    return ctr, key


def stream_words(seed: int, sid: int, first: int, count: int) -> np.ndarray:
    """Raw 32-bit words of elements [first, first + count) of stream (seed, sid)."""
    if count <= 0:
        return np.zeros(0, dtype=np.uint32)
    g0, g1 = first // 4, (first + count - 1) // 4
    ctr, key = stream_counters(seed, sid, np.arange(g0, g1 + 1, dtype=np.int64))
    words = philox4x32_10(ctr, key).reshape(-1)
    off = first - 4 * g0
    return words[off:off + count]


def open_uniform(words: np.ndarray) -> np.ndarray:
    """u = (floor(w / 2^9) + 1/2) 2^-23, in (0, 1)."""
    w = np.asarray(words, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(u1: np.ndarray, u2: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The Box-Muller pair (cosine branch, sine branch) of uniforms u1, u2."""
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)


def stream_gaussian(seed: int, sid: int, first: int, count: int) -> np.ndarray:
    """N(0, 1) values of elements [first, first + count) of stream (seed, sid)."""
    if count <= 0:
        return np.zeros(0)
    g0, g1 = first // 4, (first + count - 1) // 4
    ctr, key = stream_counters(seed, sid, np.arange(g0, g1 + 1, dtype=np.int64))
    w = philox4x32_10(ctr, key)
    u = open_uniform(w)
    z = np.empty(w.shape)
    z[:, 0], z[:, 1] = box_muller(u[:, 0], u[:, 1])
    z[:, 2], z[:, 3] = box_muller(u[:, 2], u[:, 3])
    z = z.reshape(-1)
    off = first - 4 * g0
    return z[off:off + count]


def omega(n: int, ell: int, seed: int) -> np.ndarray:
    """The raw Gaussian test matrix (n x ell, row-major) that Algorithm 1 in
    the library draws from ``seed`` when no Omega is passed in."""
    return stream_gaussian(seed, STREAM_OMEGA, 0, n * ell).reshape(n, ell)
