"""PSA+ builds (wrs_table_build_psa_plus) vs the oracle's PSA+, bucket for
bucket, through the C ABI.

Sec. 4.2 "Performance Optimization in Practice": every tile of 2048 items
first runs Alg. 2 locally in the global units until the next item it needs
lies outside the tile; the leftovers are built by Alg. 2 as one list.  The
GPU table must equal the oracle's (thresholds, aliases), the number of
leftovers must equal the oracle's, and samples drawn from the table must equal
the oracle's queries of its own table.  Sizes span several tiles with ragged
tails; the larger cases give leftover lists of many 2048-step merge blocks.
"""
import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs
from tests import _gpu as G

pytestmark = pytest.mark.gpu

TILE = 2048


def _cases():
    rng = np.random.default_rng(77)
    cases = []
    for n in (1, 2, 3, 17, TILE - 1, TILE, TILE + 1, 2 * TILE + 5, 3 * TILE + 17, 100_003):
        cases.append((f"u32_uniform_{n}", WL.u32_uniform(n, n)))
        cases.append((f"f32_uniform_{n}", WL.f32_uniform(n, n + 1)))
        cases.append((f"zipf1_{n}", WL.f32_zipf(n, 1.0, n + 2)))
    for s in (0.5, 1.5, 3.0):
        cases.append((f"zipf{s}_60000", WL.f32_zipf(60_000, s, 7)))
    n = 50_000
    base = WL.u32_uniform(n, 9)
    cases.append(("sorted_asc", np.sort(base)))
    cases.append(("sorted_desc", np.sort(base)[::-1].copy()))
    cases.append(("all_equal", np.full(n, 77, np.uint32)))
    g = np.ones(n, np.uint32)
    g[n // 3] = 10_000_000
    cases.append(("one_giant", g))
    cases.append(("small_ints_with_zeros", rng.integers(0, 4, n).astype(np.uint32)))
    z = np.zeros(n, np.uint32)
    z[::97] = 5
    cases.append(("mostly_zero", z))
    cases.append(("two_values", np.where(rng.random(n) < 0.1, 9, 1).astype(np.uint32)))
    wide = (rng.random(n) * np.exp2(rng.integers(-30, 20, n))).astype(np.float32)
    cases.append(("f32_wide_range", wide))
    sub = (rng.integers(1, 1 << 23, n) * 2.0 ** -149).astype(np.float32)
    cases.append(("f32_subnormal", sub))
    heavy_first = np.concatenate([np.full(n // 10, 1000, np.uint32), np.ones(n - n // 10, np.uint32)])
    cases.append(("heavies_first", heavy_first))
    cases.append(("heavies_last", heavy_first[::-1].copy()))
    # one heavy per tile at the tile's end: every tile stops on its last heavy
    hl = np.ones(20 * TILE, np.uint32)
    hl[TILE - 1::TILE] = 3000
    cases.append(("heavy_at_each_tile_end", hl))
    # tiles alternately all light and all heavy: the greedy pass packs nothing
    alt = np.repeat(np.where(np.arange(16) % 2 == 0, 1, 50).astype(np.uint32), TILE)
    cases.append(("alternating_tiles", alt))
    return cases


CASES = _cases()


def _check(w, t, stream_id=3):
    qz = O.quantize(w)
    tab, n_left = O.psa_plus(qz, TILE, return_left=True)
    assert t.status() == wrs.OK
    info = t.info()
    assert info.Q == qz.Q and info.shift == tab.shift and info.qp == tab.Qp
    thr, alias, res = t.download()
    bad = np.nonzero((thr != tab.thr) | (alias != tab.alias))[0]
    assert bad.size == 0, (f"{bad.size} buckets differ, first {bad[:5]}: gpu {thr[bad[:3]]},{alias[bad[:3]]} "
                           f"oracle {tab.thr[bad[:3]]},{tab.alias[bad[:3]]}")
    assert not res.any()
    assert t.psa_plus_leftovers() == n_left
    return qz, tab, n_left


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_psa_plus_matches_oracle(name, w):
    n = len(w)
    with wrs.AliasTable(n) as t:
        t.build_psa_plus(G.to_device(w))
        qz, tab, _ = _check(w, t)
        k = 3 * n + 7
        got = G.gpu_samples(t, k, seed=500 + n, stream_id=2)
        assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, k, 500 + n, 2))


@pytest.mark.parametrize("dist,n", [("uniform", 3_000_007), ("zipf1.0", 3_000_007), ("zipf1.5", 3_000_007)])
def test_psa_plus_many_merge_blocks(dist, n):
    """Leftover lists of 6 * 10^4 (uniform) to 1.4 * 10^6 (Zipf 1.5) items:
    tens to hundreds of merge blocks, each starting from a global co-rank
    search over several rounds."""
    w = WL.f32_uniform(n, 41) if dist == "uniform" else WL.f32_zipf(n, float(dist[4:]), 41)
    with wrs.AliasTable(n) as t:
        t.build_psa_plus(G.to_device(w))
        qz, tab, n_left = _check(w, t)
        assert n_left > 20 * TILE
        got = G.gpu_samples(t, 2_000_000, seed=9, stream_id=1)
        assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, 2_000_000, 9, 1))


def test_psa_plus_and_psa_share_a_table_object():
    """PSA+ and PSA builds alternate on one table object; each leaves its own
    table, and the leftover count is only reported after a PSA+ build."""
    n = 5 * TILE + 3
    w = WL.f32_zipf(n, 1.2, 13)
    qz = O.quantize(w)
    _, psa_tab = O.build_table(w)
    with wrs.AliasTable(2 * n) as t:
        for _ in range(2):
            t.build_psa_plus(G.to_device(w))
            _check(w, t)
            t.build(G.to_device(w))
            thr, alias, _ = t.download()
            assert np.array_equal(thr, psa_tab.thr) and np.array_equal(alias, psa_tab.alias)
            with pytest.raises(wrs.WrsError) as e:
                t.psa_plus_leftovers()
            assert e.value.code == wrs.EINVAL
        small = WL.u32_uniform(TILE + 1, 5)
        t.build_psa_plus(G.to_device(small))
        _check(small, t)


def test_psa_plus_invalid_weights_reported():
    w = WL.f32_uniform(10_000, 3)
    w[4321] = np.nan
    with wrs.AliasTable(len(w)) as t:
        t.build_psa_plus(G.to_device(w))
        out = torch.full((64,), -7, dtype=torch.int32, device="cuda")
        t.sample(64, 1, out=out)
        torch.cuda.synchronize()
        assert (out == -7).all()
        assert t.status() == wrs.EINVAL


def test_psa_plus_unaligned_weight_pointer():
    w = WL.f32_zipf(3 * TILE + 3, 1.0, 11)
    big = torch.from_numpy(np.concatenate([np.zeros(1, np.float32), w])).cuda()
    view = big[1:]
    assert view.data_ptr() % 16 != 0
    with wrs.AliasTable(len(w)) as t:
        t.build_psa_plus(view)
        _check(w, t)
