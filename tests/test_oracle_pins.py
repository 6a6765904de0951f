"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself:
published known-answer vectors, hand-worked examples of the paper's rules,
exact rational arithmetic, invariants of an alias table (Sec. 2.2), the
identity between Alg. 3 and Alg. 2 that Sec. 4.2 states, closed forms for
special inputs, and a chi-square test of the query rule.
"""
from __future__ import annotations

import itertools
import json
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from tests import _checks as C

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table_lists(t):
    return [t.bw_int(b) for b in range(t.n)], [int(a) for a in t.alias]


def _check(w, t):
    q, Q, _ = C.exact_units(w)
    bw, al = _table_lists(t)
    C.check_alias_table(q, Q, bw, al)


# --------------------------------------------------------------- Philox ---
def test_philox_known_answers():
    g = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for v in g["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        want = tuple(int(x, 16) for x in v["out"])
        assert O.philox(ctr, key) == want


# ------------------------------------------------------------- quantize ---
def test_quantize_u32_is_identity_and_exact_sum():
    w = WL.u32_uniform(1000, 11)
    qz = O.quantize(w)
    assert qz.beta == 0
    assert qz.Q == sum(int(x) for x in w)
    assert all(qz.q_int(i) == int(w[i]) for i in range(0, 1000, 37))


def _mixed_f32(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.integers(0, 1 << 24, size=n)
    ex = rng.integers(-30, 10, size=n)
    w = (mant.astype(np.float64) * np.exp2(ex - 23)).astype(np.float32)
    w[::17] = 0.0
    w[5] = np.float32(2.0 ** -149)          # smallest subnormal
    w[6] = np.float32(np.ldexp(0x7FFFFF, -149))  # largest subnormal
    w[7] = np.float32(1.0)
    return w


def test_quantize_f32_matches_exact_rationals():
    for seed in range(4):
        w = _mixed_f32(400, seed)
        w[5] = 0.0  # keep the range inside 2^95
        w[6] = 0.0
        qz = O.quantize(w)
        q, Q, beta = C.exact_units(w)
        assert qz.beta == beta
        assert qz.Q == Q
        assert [qz.q_int(i) for i in range(len(w))] == q
        assert Fraction(qz.Q) * Fraction(2) ** qz.beta == sum(Fraction(float(x)) for x in w)


def test_quantize_subnormals_exact():
    """Subnormal weights (exponent field 0: no hidden bit, scale 2^-149)
    beside small normal ones, within the 2^95 range, against exact rationals."""
    rng = np.random.default_rng(12)
    sub = rng.integers(1, 1 << 23, size=200).astype(np.float64) * 2.0 ** -149
    nrm = rng.integers(1 << 23, 1 << 24, size=200).astype(np.float64) * 2.0 ** rng.integers(-149, -90, size=200)
    for w in (np.array([2.0 ** -149, np.ldexp(0x7FFFFF, -149), 2.0 ** -126, 2.0 ** -100], np.float32),
              np.concatenate([sub, nrm]).astype(np.float32)):
        qz = O.quantize(w)
        q, Q, beta = C.exact_units(w)
        assert (qz.beta, qz.Q) == (beta, Q)
        assert [qz.q_int(i) for i in range(len(w))] == q


def _quantize_rejections():
    for bad in (np.nan, np.inf, -1.0, -0.0):
        test_quantize_rejects_invalid(bad)
    test_quantize_rejects_all_zero_and_empty()
    test_quantize_range_limit()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1.0, -0.0])
def test_quantize_rejects_invalid(bad):
    w = np.ones(8, dtype=np.float32)
    w[3] = bad
    with pytest.raises(O.OracleError) as e:
        O.quantize(w)
    assert e.value.code == O.EINVAL


def test_quantize_rejects_all_zero_and_empty():
    for w in (np.zeros(5, np.float32), np.zeros(5, np.uint32), np.zeros(0, np.uint32)):
        with pytest.raises(O.OracleError) as e:
            O.quantize(w)
        assert e.value.code == O.EINVAL


def test_quantize_range_limit():
    # q = 1, 2^94: Q = 2^94 + 1 < 2^95 fits
    ok = np.array([2.0 ** -10, 2.0 ** 84], dtype=np.float32)
    assert O.quantize(ok).Q == 2 ** 94 + 1
    # q = 1, 2^95, 2^95: beyond the exact range; q = 1, 2^94, 2^94: each item
    # fits, the total 2^95 + 1 does not
    for w in ([2.0 ** -11, 2.0 ** 84, 2.0 ** 84], [2.0 ** -149, 2.0 ** 100], [2.0 ** -10, 2.0 ** 84, 2.0 ** 84]):
        with pytest.raises(O.OracleError) as e:
            O.quantize(np.array(w, dtype=np.float32))
        assert e.value.code == O.EOVERFLOW


# ----------------------------------------------------- hand-worked examples
def test_hand_examples():
    g = json.load(open(os.path.join(GOLD, "hand_examples.json")))
    for ex in g["examples"]:
        w = np.array(ex["w"], dtype=np.uint32)
        qz, t = O.build_table(w)
        assert qz.Q == ex["Q"], ex["name"]
        assert [list(x) for x in zip(*_table_lists(t))] == ex["sweep"], ex["name"]
        if "vose" in ex:
            tv = O.vose(qz)
            assert [list(x) for x in zip(*_table_lists(tv))] == ex["vose"], ex["name"]
        if "split" in ex:
            sp = ex["split"]
            tp, splits = O.psa(qz, sp["p"], return_splits=True)
            row = [int(x) for x in splits[1]]
            assert row == [sp["nprime"], sp["i"], sp["j"], sp["r"]], ex["name"]
    for ex in g["f32_examples"]:
        w = np.array(ex["w"], dtype=np.float32)
        qz, t = O.build_table(w)
        assert qz.beta == ex["beta"] and qz.Q == ex["Q"]
        assert [qz.q_int(i) for i in range(len(w))] == ex["q"]
        assert [list(x) for x in zip(*_table_lists(t))] == ex["sweep"], ex["name"]


def test_split_ambiguity_example_both_j_satisfy_paper_condition():
    """Alg. 3's split condition admits j = 0 and j = 1 for w = 1,3,1,3 and
    n' = 2; the oracle returns the largest (the state of Alg. 2)."""
    w = [1, 3, 1, 3]
    W, n, nprime = sum(w), 4, 2
    l = [1, 1]
    h = [3, 3]
    ok = []
    for j in range(0, 3):
        i = nprime - j
        if i < 0 or i > len(l) or j > len(h):
            continue
        sigma = sum(l[:i]) + sum(h[:j])
        nxt = h[j] if j < len(h) else float("inf")
        if Fraction(sigma) <= Fraction(nprime * W, n) < sigma + nxt:
            ok.append(j)
    assert ok == [0, 1]


# ------------------------------------------------- invariants, brute force
def _all_small_vectors():
    for n in range(1, 6):
        for w in itertools.product(range(5), repeat=n):
            if sum(w) > 0:
                yield np.array(w, dtype=np.uint32)


def test_exhaustive_small_sweep_psa_vose_are_alias_tables():
    count = 0
    for w in _all_small_vectors():
        qz, ts = O.build_table(w)
        _check(w, ts)
        _check(w, O.vose(qz))
        for p in range(1, len(w) + 1):
            tp = O.psa(qz, p)
            assert np.array_equal(tp.bw, ts.bw) and np.array_equal(tp.alias, ts.alias), (w, p)
        count += 1
    assert count == sum(5 ** n for n in range(1, 6)) - 5


def test_exact_query_distribution_equals_definition():
    """P[X = i] = w_i / W (problem WRS-1) for the table plus the query rule,
    summed in closed form over all 2^128 random bit patterns."""
    rng = random.Random(5)
    cases = [np.array(w, dtype=np.uint32) for w in ([1], [1, 3], [5, 1, 1, 5, 0, 0], [7, 7, 7])]
    cases += [np.array([rng.randrange(0, 1 << 24) for _ in range(rng.randrange(1, 11))], dtype=np.uint32)
              for _ in range(30)]
    # f32 inputs with Q >= 2^64 exercise the thr = bw >> s encoding
    cases += [np.array([2.0 ** -70, 1.0, 0.5, 2.0 ** -3], dtype=np.float32),
              np.array([2.0 ** -60 * 3, 1.5, 2.0 ** -60, 0.75, 1.0], dtype=np.float32)]
    for w in cases:
        if int(np.asarray(w, dtype=np.float64).sum()) == 0 and w.dtype == np.uint32 and w.sum() == 0:
            continue
        q, Q, _ = C.exact_units(w)
        qz, t = O.build_table(w)
        n = len(w)
        p = C.exact_query_distribution(t.thr, t.alias, t.Qp)
        bound = Fraction(4 * n, 1 << 64)
        if t.shift:
            bound += Fraction(4 * n * (1 << t.shift), Q)
        for i in range(n):
            assert abs(p[i] - Fraction(q[i], Q)) <= bound, (w, i, float(p[i]), q[i] / Q)


def test_random_tables_invariants_and_psa_identity():
    rng = np.random.default_rng(9)
    for trial in range(40):
        n = int(rng.integers(1, 3000))
        kind = trial % 4
        if kind == 0:
            w = WL.u32_uniform(n, trial)
        elif kind == 1:
            w = WL.f32_uniform(n, trial)
        elif kind == 2:
            w = WL.f32_zipf(n, [0.5, 1.0, 1.5, 2.0][trial % 4], trial)
        else:
            w = rng.integers(0, 4, size=n).astype(np.uint32)
            if w.sum() == 0:
                w[0] = 1
        qz, ts = O.build_table(w)
        _check(w, ts)
        for p in {1, 2, 3, 64, n, int(rng.integers(1, n + 1))}:
            if p > n:
                continue
            tp = O.psa(qz, p)
            assert np.array_equal(tp.bw, ts.bw) and np.array_equal(tp.alias, ts.alias), (trial, p)


def test_psa_splits_satisfy_paper_condition():
    """Every split (i, j, spill) meets Alg. 3's condition sigma <= n'W/n <
    sigma + w_{h[j+1]}, i + j = n', and spill = w_{h[j+1]} + sigma - n'W/n,
    checked with exact rationals on the raw weights."""
    for trial in range(12):
        n = 50 + 37 * trial
        w = WL.f32_zipf(n, 1.0, trial) if trial % 2 else WL.u32_uniform(n, trial)
        fr = [Fraction(float(x)) for x in w] if w.dtype == np.float32 else [Fraction(int(x)) for x in w]
        W = sum(fr)
        light = [x for x in fr if x <= W / n]
        heavy = [x for x in fr if x > W / n]
        q, Q, beta = C.exact_units(w)
        scale = Fraction(n) / Fraction(2) ** beta  # paper units -> scaled integer units
        p = 1 + trial % 9
        qz = O.quantize(w)
        _, splits = O.psa(qz, p, return_splits=True)
        for k in range(1, p):
            nprime, i, j, r = (int(x) for x in splits[k])
            assert nprime == -(-n * k // p) and i + j == nprime
            sigma = sum(light[:i]) + sum(heavy[:j])
            target = Fraction(nprime) * W / n
            assert sigma <= target
            if j < len(heavy):
                assert sigma + heavy[j] > target
                assert Fraction(r) == (heavy[j] + sigma - target) * scale
            # no larger j satisfies the condition (the reading: largest j)
            if j + 1 <= min(nprime, len(heavy)) and nprime - j - 1 >= 0:
                s2 = sum(light[:i - 1]) + sum(heavy[:j + 1])
                assert s2 > target


# ---------------------------------------------------------- special cases
def test_all_equal_weights_give_full_self_buckets():
    for n in (1, 2, 7, 1000):
        for w in (np.full(n, 5, np.uint32), np.full(n, 0.3, np.float32)):
            qz, t = O.build_table(w)
            assert all(t.bw_int(b) == qz.Q for b in range(n))
            assert np.array_equal(t.alias, np.arange(n, dtype=np.uint32))
            assert np.all(t.thr == t.Qp)


def test_one_heavy_among_equal_lights_closed_form():
    """Heavy H at position p among n-1 lights of weight c < H: every light
    bucket holds n*c with alias p; the heavy bucket ends exactly full."""
    for n, H, c, pos in ((5, 9, 2, 0), (9, 100, 3, 4), (64, 1000, 1, 63), (10, 7, 0, 2)):
        w = np.full(n, c, np.uint32)
        w[pos] = H
        qz, t = O.build_table(w)
        Q = H + (n - 1) * c
        assert qz.Q == Q
        for b in range(n):
            if b == pos:
                assert t.bw_int(b) == Q and t.alias[b] == pos
            else:
                assert t.bw_int(b) == n * c and t.alias[b] == pos


def test_two_items_closed_form():
    for a, b in ((1, 3), (3, 1), (0, 5), (4, 4), (1, 1 << 31)):
        w = np.array([a, b], np.uint32)
        qz, t = O.build_table(w)
        Q = a + b
        got = list(zip(*_table_lists(t)))
        if a < b:
            assert got == [(2 * a, 1), (Q, 1)]
        elif a > b:
            assert got == [(Q, 0), (2 * b, 0)]
        else:
            assert got == [(Q, 0), (Q, 1)]


def test_vose_f64_against_exact_probabilities():
    for seed in range(3):
        w = WL.f32_uniform(5000, seed)
        prob, al = O.vose_f64(w.astype(np.float64))
        n = len(w)
        mass = np.zeros(n)
        np.add.at(mass, np.arange(n), prob)
        other = al != np.arange(n)
        np.add.at(mass, al[other], 1.0 - prob[other])
        q, Q, _ = C.exact_units(w)
        p_exact = np.array([Fraction(x, Q) for x in q], dtype=np.float64)
        rel = np.abs(mass / n - p_exact) / p_exact
        assert rel.max() < 1e-9


# ---------------------------------------------------------------- sampler
def test_sampler_n1_and_full_buckets_reduce_to_multiply_shift():
    assert np.all(O.sample(np.array([7], np.uint64), np.array([0], np.uint32), 7, 100, 3) == 0)
    n = 1000
    w = np.full(n, 9, np.uint32)
    qz, t = O.build_table(w)
    out = O.sample(t.thr, t.alias, t.Qp, 500, seed=42, stream=7)
    for s in range(500):
        x = O.philox([s & 0xFFFFFFFF, s >> 32, 7, 0], [42, 0])
        u = x[0] | (x[1] << 32)
        assert out[s] == (u * n) >> 64  # Lemire's multiply-shift bucket choice


def test_closed_form_counts_match_brute_force():
    """The closed forms behind the exact query distribution, checked by
    counting every word of a 12-bit analogue: how many u pick bucket r under
    multiply-shift (always floor or ceil of 2^bits / n), and how many v pass
    the coin floor(v * Qp / 2^bits) < thr."""
    bits = 12
    u = np.arange(1 << bits, dtype=np.int64)
    for n in list(range(1, 130)) + [1000, 4095, 4096]:
        got = np.bincount((u * n) >> bits, minlength=n)
        want = [C.bucket_count(r, n, bits) for r in range(n)]
        assert got.tolist() == want, n
        assert set(want) <= {(1 << bits) // n, -(-(1 << bits) // n)}, n
    for Qp in (1, 2, 3, 7, 100, 4095, 4096, 5000):
        for thr in sorted({0, 1, 2, Qp // 3, Qp // 2, Qp - 1, Qp, Qp + 1}):
            assert int(((u * Qp) >> bits < thr).sum()) == C.coin_heads(thr, Qp, bits), (Qp, thr)
    # at the full width every bucket count is still floor or ceil of 2^64 / n
    for n in (3, 10 ** 6, 10 ** 9, 2 ** 32 - 1):
        lo, hi = (1 << 64) // n, -(-(1 << 64) // n)
        for r in (0, 1, n // 2, n - 1):
            assert C.bucket_count(r, n) in (lo, hi)


def test_sampler_tails_take_the_alias():
    n = 37
    thr = np.zeros(n, np.uint64)
    alias = ((np.arange(n) + 1) % n).astype(np.uint32)
    out = O.sample(thr, alias, 1 << 40, 300, seed=1)
    for s in range(300):
        x = O.philox([s, 0, 0, 0], [1, 0])
        r = ((x[0] | (x[1] << 32)) * n) >> 64
        assert out[s] == (r + 1) % n


def test_sampler_coin_with_small_denominator():
    """Two buckets, bucket 0 full, bucket 1 holding thr/qp of itself and item
    0 as alias: P[X = 1] = (1/2) * (thr/qp) exactly (each bucket is drawn
    with probability 1/2 since 2^64 is even; the coin is heads with
    probability ceil(thr * 2^64 / qp) / 2^64)."""
    k = 200_000
    for qp, t1 in ((2, 1), (3, 1), (3, 2), (7, 3)):
        thr = np.array([qp, t1], np.uint64)
        alias = np.array([0, 0], np.uint32)
        out = O.sample(thr, alias, qp, k, seed=11 + qp, stream=t1)
        p1 = 0.5 * C.coin_heads(t1, qp) / 2 ** 64
        hits = int((out == 1).sum())
        sd = (k * p1 * (1 - p1)) ** 0.5
        assert abs(hits - k * p1) < 6 * sd, (qp, t1, hits, k * p1)


def test_sampler_chi_square():
    from scipy import stats
    w = WL.f32_zipf(200, 1.0, 3)
    qz, t = O.build_table(w)
    k = 2_000_000
    out = O.sample(t.thr, t.alias, t.Qp, k, seed=2024, stream=1)
    counts = np.bincount(out, minlength=len(w))
    p = np.array([qz.q_int(i) for i in range(len(w))], dtype=np.float64) / float(qz.Q)
    chi2 = float(((counts - k * p) ** 2 / (k * p)).sum())
    df = len(w) - 1
    z = (chi2 - df) / np.sqrt(2 * df)
    assert abs(z) < 5, z
    assert stats.chi2.sf(chi2, df) > 1e-6


def test_sampler_streams_and_seeds():
    w = WL.u32_uniform(1000, 4)
    qz, t = O.build_table(w)
    a = O.sample(t.thr, t.alias, t.Qp, 1000, seed=5, stream=0)
    b = O.sample(t.thr, t.alias, t.Qp, 1000, seed=5, stream=0)
    c = O.sample(t.thr, t.alias, t.Qp, 1000, seed=5, stream=1)
    d = O.sample(t.thr, t.alias, t.Qp, 1000, seed=6, stream=0)
    assert np.array_equal(a, b)
    assert (a != c).mean() > 0.9 and (a != d).mean() > 0.9


# ------------------------------------------------------------- generators
def test_permutation_is_bijection():
    for n in (1, 2, 3, 1000, 65536, 100_003):
        p = WL.permutation(n, 7)
        assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint64))


def test_generators_ranges_and_determinism():
    u = WL.u32_uniform(10000, 1)
    assert u.min() >= 1 and u.max() <= 1 << 24
    f = WL.f32_uniform(10000, 3)
    assert f.min() > 0 and f.max() <= 1.0
    assert np.all((f.astype(np.float64) * 2 ** 24) == np.round(f.astype(np.float64) * 2 ** 24))
    z = WL.f32_zipf(10000, 1.0, 4)
    assert np.isclose(np.sort(z)[::-1][:3].astype(np.float64), [1.0, 0.5, 1 / 3]).all()
    assert np.array_equal(WL.u32_uniform(100, 1), u[:100])
