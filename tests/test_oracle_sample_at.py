"""Pins of the oracle's indexed queries (``sample_at``, ``sample_2lvl_at``),
the checkers of every full-size sample test.

Two kinds of pins, neither of which reuses the helpers' own code:
* consistency with the sequential samplers (``sample``, ``sample_2lvl``,
  themselves pinned by the exact query distribution and the two-level
  probabilities) on random and edge indices, with stream ids >= 2^32;
* for counters and keys whose high words are set (sample index >= 2^32), the
  published Philox4x32-10 known-answer vectors (Salmon et al., SC'11): a
  table whose buckets are all full returns Lemire's multiply-shift of the
  published low word, one whose buckets are all empty returns the alias of
  that bucket, and a coin threshold splits on the published high word (the
  query of Sec. 2.2).
"""
import json
import os

import numpy as np

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")
W0, W1 = 0x9E3779B9, 0xBB67AE85
M64 = (1 << 64) - 1


def _kat():
    with open(GOLDEN) as f:
        vecs = json.load(f)["vectors"]
    out = []
    for v in vecs:
        c = [int(x, 16) for x in v["ctr"]]
        k = [int(x, 16) for x in v["key"]]
        o = [int(x, 16) for x in v["out"]]
        out.append((c, k, o))
    return out


def _edge_indices(k, rng, m=200):
    idx = set(rng.integers(0, k, size=m).tolist()) | {0, 1, k // 2, k - 2, k - 1}
    return np.array(sorted(idx), dtype=np.uint64)


def test_sample_at_equals_sequential_queries():
    rng = np.random.default_rng(17)
    for w, seed, stream in ((WL.f32_zipf(3001, 1.0, 2), 0x1234_5678_9ABC_DEF0, (1 << 33) + 5),
                            (WL.u32_uniform(777, 3), 99, 0),
                            (WL.f32_uniform(64, 4), (1 << 63) + 7, (1 << 64) - 1)):
        qz, t = O.build_table(w)
        k = 5000
        full = O.sample(t.thr, t.alias, t.Qp, k, seed, stream)
        idx = _edge_indices(k, rng)
        got = O.sample_at(t.thr, t.alias, t.Qp, seed, stream, idx)
        assert np.array_equal(got, full[idx.astype(np.int64)])


def test_sample_at_high_counter_words_against_published_philox():
    """Sample index s = ctr0 | ctr1 << 32 (>= 2^32 for two of the vectors),
    stream = ctr2 | ctr3 << 32, seed = key0 | key1 << 32: the published
    output gives u (low 64 bits) and v (high 64 bits)."""
    n = 1009
    alias = ((np.arange(n) * 7 + 3) % n).astype(np.uint32)
    for c, key, o in _kat():
        s = c[0] | (c[1] << 32)
        stream = c[2] | (c[3] << 32)
        seed = key[0] | (key[1] << 32)
        u = o[0] | (o[1] << 32)
        v = o[2] | (o[3] << 32)
        r = (u * n) >> 64
        idx = np.array([s], dtype=np.uint64)
        # every bucket full (threshold = denominator): heads, the bucket itself
        qp = 1 << 63
        thr = np.full(n, qp, np.uint64)
        assert O.sample_at(thr, alias, qp, seed, stream, idx)[0] == r
        # every bucket empty: the alias of the bucket
        thr0 = np.zeros(n, np.uint64)
        assert O.sample_at(thr0, alias, qp, seed, stream, idx)[0] == alias[r]
        # a coin exactly at the published word: heads iff floor(v * qp / 2^64) < thr
        for qp2 in (3, 1000, (1 << 64) - 59):
            coin = (v * qp2) >> 64
            for t in (coin, coin + 1):
                thr1 = np.full(n, min(t, qp2), np.uint64)
                want = r if coin < min(t, qp2) else alias[r]
                assert O.sample_at(thr1, alias, qp2, seed, stream, idx)[0] == want, (qp2, t)
        # the sequential sampler agrees where it can reach the counter (s < 2^32)
        if s < (1 << 32) and s < 4096:
            full = O.sample(thr0, alias, qp, s + 1, seed, stream)
            assert full[s] == alias[r]


def test_sample_2lvl_at_equals_sequential_walk():
    rng = np.random.default_rng(5)
    for n, G, seed, stream in ((5000, 16, 0xDEAD_BEEF_0000_0001, (1 << 40) + 3),
                               (3000, 2048, 12, 1),
                               (700, 3, (1 << 64) - 2, 0)):
        qz = O.quantize(WL.f32_zipf(n, 0.9, 8))
        t = O.build_2lvl(qz, G)
        k = 4000
        full = O.sample_2lvl(t, k, seed, stream)
        idx = _edge_indices(k, rng)
        got = O.sample_2lvl_at(t, seed, stream, idx)
        assert np.array_equal(got, full[idx.astype(np.int64)]), (n, G)


def test_sample_2lvl_at_bottom_level_against_published_philox():
    """Two levels of all-equal weights (every bucket full, at both levels):
    the top draw (key = seed) names group g, the bottom draw (key = seed +
    the Weyl constants) picks member floor(u * n_g / 2^64) of it.  The seed
    is chosen so that the bottom draw's key is a published vector's key, so
    its u is the published low word."""
    G = 10
    ngroups = 7
    n = G * ngroups
    qz = O.quantize(np.full(n, 5, np.uint32))
    t = O.build_2lvl(qz, G)
    assert t.levels == 2
    for c, key, o in _kat():
        s = c[0] | (c[1] << 32)
        stream = c[2] | (c[3] << 32)
        seed = ((key[0] - W0) & 0xFFFFFFFF) | (((key[1] - W1) & 0xFFFFFFFF) << 32)
        top = O.philox(c, [seed & 0xFFFFFFFF, seed >> 32])
        g = ((top[0] | (top[1] << 32)) * ngroups) >> 64
        u = o[0] | (o[1] << 32)
        want = g * G + ((u * G) >> 64)
        got = O.sample_2lvl_at(t, seed, stream, np.array([s], dtype=np.uint64))[0]
        assert got == want, (hex(s), got, want)
