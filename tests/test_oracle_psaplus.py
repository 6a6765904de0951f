"""Pins of the oracle's PSA+ (Sec. 4.2 "Performance Optimization in
Practice": greedy per-tile packing, then PSA on what is left), against facts
independent of its code: with one-item tiles or one tile holding everything
it is exactly Alg. 2 (pinned elsewhere); for every tile size its table is an
alias table of the weights (Sec. 2.2 definition, checked exactly); on random
uniform inputs the greedy phase leaves few items."""
import itertools

import numpy as np
import pytest

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from tests import _checks as C


def _inputs():
    rng = np.random.default_rng(3)
    out = [("zipf1", WL.f32_zipf(7000, 1.0, 3)), ("zipf1.5", WL.f32_zipf(7000, 1.5, 4)),
           ("uniform", WL.f32_uniform(7000, 5)), ("u32", WL.u32_uniform(5000, 6))]
    base = WL.u32_uniform(4000, 7)
    out.append(("sorted_asc", np.sort(base)))
    out.append(("sorted_desc", np.sort(base)[::-1].copy()))
    out.append(("all_equal", np.full(3000, 5, np.uint32)))
    g = np.ones(3000, np.uint32)
    g[1234] = 10 ** 7
    out.append(("one_giant", g))
    out.append(("zeros", rng.integers(0, 3, 3000).astype(np.uint32)))
    return out


INPUTS = _inputs()


@pytest.mark.parametrize("name,w", INPUTS, ids=[x[0] for x in INPUTS])
def test_degenerate_tile_sizes_are_alg2(name, w):
    qz, ref = O.build_table(w)
    for T in (1, len(w), 10 ** 9):
        t = O.psa_plus(qz, T)
        assert np.array_equal(t.thr, ref.thr) and np.array_equal(t.alias, ref.alias), T


@pytest.mark.parametrize("name,w", INPUTS, ids=[x[0] for x in INPUTS])
@pytest.mark.parametrize("T", [2, 3, 7, 64, 2048])
def test_every_tile_size_gives_an_alias_table(name, w, T):
    qz = O.quantize(w)
    t = O.psa_plus(qz, T)
    C.check_alias_table([qz.q_int(i) for i in range(qz.n)], qz.Q, [t.bw_int(b) for b in range(qz.n)],
                        [int(a) for a in t.alias])


def test_exhaustive_small():
    for n in range(1, 6):
        for ws in itertools.product(range(4), repeat=n):
            if sum(ws) == 0:
                continue
            w = np.array(ws, dtype=np.uint32)
            qz = O.quantize(w)
            for T in (1, 2, 3):
                t = O.psa_plus(qz, T)
                C.check_alias_table(list(ws), int(sum(ws)), [t.bw_int(b) for b in range(n)],
                                    [int(a) for a in t.alias])


def test_greedy_phase_leaves_few_items_on_uniform_inputs():
    qz = O.quantize(WL.f32_uniform(200_000, 9))
    _, left = O.psa_plus(qz, 2048, return_left=True)
    assert left < 0.05 * qz.n


def test_hand_examples():
    """Tables worked by hand from the PSA+ rule (tests/golden/
    psa_plus_hand_examples.json): buckets, leftover count, and, for the first
    example, a table different from Alg. 2's on the same weights."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "psa_plus_hand_examples.json")))
    for ex in g["examples"]:
        w = np.array(ex["w"], np.uint32)
        qz = O.quantize(w)
        assert qz.Q == ex["Q"]
        t, n_left = O.psa_plus(qz, ex["T"], return_left=True)
        want = np.array(ex["psa_plus"], np.uint64)
        assert np.array_equal(t.thr, want[:, 0]) and np.array_equal(t.alias, want[:, 1].astype(np.uint32)), ex["name"]
        assert n_left == ex["n_left"]
        _, ref = O.build_table(w)
        a2 = np.array(ex["alg2"], np.uint64)
        assert np.array_equal(ref.thr, a2[:, 0]) and np.array_equal(ref.alias, a2[:, 1].astype(np.uint32))
    assert g["examples"][0]["psa_plus"] != g["examples"][0]["alg2"]
