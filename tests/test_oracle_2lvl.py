"""Pins of the oracle's two-level ("2lvl-sweep") tables (Sec. 6 with the
replicated top level, Alg. 2 per group), against facts that do not come from
the oracle's own code:

* with one group (n <= G) the structure is exactly Alg. 2's table and its
  samples exactly the single-table queries (both pinned elsewhere);
* every group's table is an alias table of its members in the group's own
  units (Sec. 2.2 definition, checked independently);
* the probability of every item under the sampling rule, summed in closed
  form over all random words at every level, equals w_i / W up to the
  discretisation bound -- on tiny group sizes that make three and more
  levels, and on the library's group size;
* the level sizes follow ceil(n / G) to a single group.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from tests import _checks as C


def _groups(t, level):
    """(first member, member count) of every group of a level."""
    N, G = t.sizes[level], t.G
    return [(b, min(G, N - b)) for b in range(0, N, G)]


def _level_weights(q_ints, t):
    """Exact member weights of every level: the items, then group totals."""
    out = [list(q_ints)]
    for level in range(1, t.levels):
        prev = out[-1]
        out.append([sum(prev[b:b + m]) for b, m in _groups(t, level - 1)])
    return out


def test_hand_examples():
    """Two-level tables worked by hand (tests/golden/two_level_hand_examples.json):
    three levels of groups of two, with and without zero weights."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "two_level_hand_examples.json")))
    for ex in g["examples"]:
        qz = O.quantize(np.array(ex["w"], np.uint32))
        t = O.build_2lvl(qz, ex["G"])
        assert list(t.sizes) == ex["levels"], ex["name"]
        assert t.thr.tolist() == ex["thr"], ex["name"]
        assert t.alias.tolist() == ex["alias"], ex["name"]
        assert t.qp.tolist() == ex["qp"] and not t.shift.any(), ex["name"]


def test_level_sizes():
    assert O.levels_2lvl(1) == [1]
    assert O.levels_2lvl(2048) == [2048]
    assert O.levels_2lvl(2049) == [2049, 2]
    assert O.levels_2lvl(2048 * 2048) == [2048 * 2048, 2048]
    assert O.levels_2lvl(2048 * 2048 + 1) == [2048 * 2048 + 1, 2049, 2]
    assert O.levels_2lvl(10 ** 9) == [10 ** 9, 488282, 239]
    assert O.levels_2lvl(7, 2) == [7, 4, 2]


@pytest.mark.parametrize("n", [1, 2, 3, 100, 2047, 2048])
def test_single_group_is_alg2(n):
    for w in (WL.f32_zipf(n, 1.0, n), WL.u32_uniform(n, n + 1)):
        qz, tab = O.build_table(w)
        t = O.build_2lvl(qz)
        assert t.levels == 1
        assert np.array_equal(t.thr, tab.thr) and np.array_equal(t.alias, tab.alias)
        assert int(t.qp[0]) == tab.Qp and int(t.shift[0]) == tab.shift
        assert np.array_equal(O.sample_2lvl(t, 3000, 9, 4), O.sample(tab.thr, tab.alias, tab.Qp, 3000, 9, 4))


GROUP_CASES = [(7, 2, 1), (30, 3, 2), (100, 4, 3), (5000, 2048, 4), (9000, 64, 5)]
PROB_CASES = [(7, 2, 11), (13, 3, 12), (40, 4, 13), (3000, 2048, 14)]


@pytest.mark.parametrize("n,G,seed", GROUP_CASES)
def test_every_group_is_an_alias_table(n, G, seed):
    w = WL.u32_uniform(n, seed)
    w[::7] = 0  # zero weights: light, never sampled
    qz = O.quantize(w)
    t = O.build_2lvl(qz, G)
    weights = _level_weights([qz.q_int(i) for i in range(n)], t)
    for level in range(t.levels):
        ls, gs = t.level_slice(level), t.group_slice(level)
        thr, al = t.thr[ls], t.alias[ls]
        for gi, (b, m) in enumerate(_groups(t, level)):
            qg = weights[level][b:b + m]
            Qg = sum(qg)
            assert O.u128_to_int(t.tot[gs][gi]) == Qg
            assert int(t.shift[gs][gi]) == 0 and int(t.qp[gs][gi]) == Qg  # Q_g < 2^64 here
            # in the group's units a member weighs m * q; with shift 0, thr is the exact bw
            C.check_alias_table(qg, Qg, [int(x) for x in thr[b:b + m]], [int(a) - b for a in al[b:b + m]])


def _exact_item_probabilities(t):
    """P[sample = i] under the sampling rule: product over levels of the exact
    single-group query distribution of the member taken at that level."""
    per_level = []
    for level in range(t.levels):
        ls, gs = t.level_slice(level), t.group_slice(level)
        thr, al = t.thr[ls], t.alias[ls]
        p = [Fraction(0)] * t.sizes[level]
        for gi, (b, m) in enumerate(_groups(t, level)):
            local = C.exact_query_distribution(thr[b:b + m], [int(a) - b for a in al[b:b + m]], int(t.qp[gs][gi]))
            for j in range(m):
                p[b + j] = local[j]
        per_level.append(p)
    probs = []
    for i in range(t.n):
        pr, idx = Fraction(1), i
        for level in range(t.levels):
            pr *= per_level[level][idx]
            idx //= t.G
        probs.append(pr)
    return probs


@pytest.mark.parametrize("n,G,seed", PROB_CASES)
def test_item_probabilities_are_the_weights(n, G, seed):
    w = WL.f32_zipf(n, 1.2, seed)
    w[3] = 0.0
    qz = O.quantize(w)
    t = O.build_2lvl(qz, G)
    probs = _exact_item_probabilities(t)
    Q = qz.Q
    bound = Fraction(8 * t.levels * G, 2 ** 64)  # bucket choice and coin per level
    for i in range(n):
        target = Fraction(qz.q_int(i), Q)
        assert abs(probs[i] - target) <= bound * max(target, Fraction(1, n * n)) + Fraction(4 * G, 2 ** 64), i
    assert probs[3] == 0  # a zero weight is never drawn
    assert sum(probs) == 1


def test_samples_follow_the_weights():
    n, k = 5000, 400_000
    w = WL.f32_zipf(n, 1.0, 21)
    qz = O.quantize(w)
    t = O.build_2lvl(qz, 64)  # three levels
    assert t.levels == 3
    s = O.sample_2lvl(t, k, 3, 1)
    cnt = np.bincount(s, minlength=n).astype(np.float64)
    p = np.array([qz.q_int(i) for i in range(n)], dtype=np.float64) / float(qz.Q)
    e = k * p
    keep = e >= 5
    chi2 = float(((cnt[keep] - e[keep]) ** 2 / e[keep]).sum()) + float(
        (cnt[~keep].sum() - e[~keep].sum()) ** 2 / max(e[~keep].sum(), 1e-9))
    dof = int(keep.sum())
    assert abs(chi2 - dof) < 6 * np.sqrt(2 * dof), (chi2, dof)
    at = O.sample_2lvl_at(t, 3, 1, np.array([0, 17, k - 1], dtype=np.uint64))
    assert list(at) == [s[0], s[17], s[k - 1]]
