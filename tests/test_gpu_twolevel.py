"""Two-level ("2lvl-sweep") tables on the GPU vs the CPU oracle, bit for bit:
buckets of every level, group records and samples, for one to three levels,
ragged groups, both word types, the paper's shapes and degenerate inputs."""
import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs

pytestmark = pytest.mark.gpu

G = 2048


def _cases():
    cases = []
    for n in (1, 2, 17, G - 1, G, G + 1, 3 * G + 5, 100_003):
        cases.append((f"u32_{n}", WL.u32_uniform(n, n)))
        cases.append((f"f32_{n}", WL.f32_uniform(n, n + 1)))
        cases.append((f"zipf1_{n}", WL.f32_zipf(n, 1.0, n + 2)))
    for s in (0.8, 1.5, 3.0):
        cases.append((f"zipf{s}_70000", WL.f32_zipf(70_000, s, 4)))
    rng = np.random.default_rng(5)
    z = np.zeros(50_000, np.uint32)
    z[::97] = 5
    cases.append(("mostly_zero", z))
    zg = WL.u32_uniform(5 * G, 6)
    zg[G:2 * G] = 0  # a whole group of zeros
    cases.append(("zero_group", zg))
    g1 = np.ones(30_000, np.uint32)
    g1[12_345] = 10_000_000
    cases.append(("one_giant", g1))
    cases.append(("all_equal", np.full(9000, 3, np.uint32)))
    wide = (rng.random(40_000) * np.exp2(rng.integers(-30, 20, 40_000))).astype(np.float32)
    cases.append(("f32_wide_range", wide))
    return cases


CASES = _cases()


def _check(w, t2, k=20_000, seed=3, sid=7):
    qz = O.quantize(w)
    ref = O.build_2lvl(qz)
    assert t2.status() == wrs.OK
    assert t2.levels() == ref.sizes
    thr, alias, res, qp, shift, members = t2.download()
    bad = np.nonzero((thr != ref.thr) | (alias != ref.alias))[0]
    assert bad.size == 0, f"{bad.size} buckets differ, first {bad[:5]}"
    assert not res.any()
    assert np.array_equal(qp, ref.qp) and np.array_equal(shift, ref.shift)
    gm = [min(G, m - b) for m in ref.sizes for b in range(0, m, G)]
    assert list(members) == gm
    out = t2.sample(k, seed, sid)
    torch.cuda.synchronize()
    got = out[:k].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, O.sample_2lvl(ref, k, seed, sid))


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_two_level_matches_oracle(name, w):
    wt = torch.from_numpy(w.view(np.int32).copy() if w.dtype == np.uint32 else w.copy()).cuda()
    with wrs.AliasTable2(len(w)) as t2:
        t2.build(wt)
        _check(w, t2)


def test_three_levels():
    n = G * G + 4099  # 2050 groups at level 1, two at level 2
    w = WL.f32_zipf(n, 1.0, 8)
    with wrs.AliasTable2(n) as t2:
        t2.build(torch.from_numpy(w).cuda())
        assert len(t2.levels()) == 3
        _check(w, t2, k=200_000)


def test_one_group_equals_single_table():
    w = WL.f32_zipf(1500, 1.2, 9)
    with wrs.AliasTable(1500) as a, wrs.AliasTable2(1500) as b:
        a.build(torch.from_numpy(w).cuda())
        b.build(torch.from_numpy(w).cuda())
        ta, aa, _ = a.download()
        tb, ab, *_ = b.download()
        assert np.array_equal(ta, tb) and np.array_equal(aa, ab)
        sa = a.sample(10_000, 4, 2).cpu().numpy()
        sb = b.sample(10_000, 4, 2).cpu().numpy()
        assert np.array_equal(sa, sb)


def test_rebuild_and_errors():
    with wrs.AliasTable2(3 * G) as t2:
        for seed, n in ((1, 3 * G), (2, 10), (3, 2 * G + 1)):
            w = WL.f32_zipf(n, 1.0, seed)
            t2.build(torch.from_numpy(w).cuda())
            _check(w, t2, k=1000)
        bad = WL.f32_uniform(2 * G, 4)
        bad[77] = np.nan
        t2.build(torch.from_numpy(bad).cuda())
        out = torch.full((100,), -7, dtype=torch.int32, device="cuda")
        wrs.table2_sample(t2.handle, 100, 1, 0, out.data_ptr(), 0)
        torch.cuda.synchronize()
        assert (out == -7).all()
        assert t2.status() == wrs.EINVAL
    rc, _ = wrs.table2_create(0)
    assert rc == wrs.EINVAL
