"""OS-ND output-sensitive sampling on the GPU vs the CPU oracle: the same
(item, count) pairs (as a multiset: the GPU writes them in no fixed order)
for one to three levels, base-case and descent regimes, k from 1 to 10^12."""
import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs

pytestmark = pytest.mark.gpu


def _sorted_pairs(items, counts):
    items = np.asarray(items, dtype=np.uint64)
    counts = np.asarray(counts, dtype=np.uint64)
    order = np.lexsort((counts, items))
    return items[order], counts[order]


def _run(w, ks, seed=5, stream=3):
    wt = torch.from_numpy(w.view(np.int32).copy() if w.dtype == np.uint32 else w.copy()).cuda()
    qz = O.quantize(w)
    ref = O.build_2lvl(qz)
    with wrs.AliasTable2(len(w)) as t2:
        t2.build(wt)
        assert t2.status() == wrs.OK
        for k in ks:
            gi, gc = t2.sample_os(wt, k, seed, stream)
            got = _sorted_pairs(gi.cpu().numpy().view(np.uint32), gc.cpu().numpy().view(np.uint64))
            want = _sorted_pairs(*O.os_nd(qz, ref, k, seed, stream))
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), k
            assert int(got[1].sum()) == k


@pytest.mark.parametrize("name,w", [
    ("zipf1.2_5000", WL.f32_zipf(5000, 1.2, 3)),
    ("zipf1.5_100003", WL.f32_zipf(100_003, 1.5, 4)),
    ("uniform_1000", WL.f32_uniform(1000, 5)),
    ("u32_70000", WL.u32_uniform(70_000, 6)),
], ids=lambda x: x if isinstance(x, str) else None)
def test_osnd_matches_oracle(name, w):
    _run(w, [1, 50, 127, 128, 1000, 10 ** 6, 10 ** 9, 10 ** 12])


def test_osnd_three_levels():
    n = 2048 * 2048 + 4099
    _run(WL.f32_zipf(n, 1.5, 8), [100, 10 ** 6, 10 ** 9])


def test_osnd_capacity_and_arguments():
    w = WL.f32_zipf(20_000, 1.0, 9)
    wt = torch.from_numpy(w).cuda()
    with wrs.AliasTable2(len(w)) as t2:
        t2.build(wt)
        with pytest.raises(wrs.WrsError):
            t2.sample_os(wt, 10 ** 6, 1, 0, capacity=10)
        ints = torch.from_numpy(WL.u32_uniform(20_000, 1).view(np.int32)).cuda()
        with pytest.raises(wrs.WrsError):
            t2.sample_os(ints, 100, 1, 0)  # the table was built from binary32 words
        items, counts = t2.sample_os(wt, 0, 1, 0)
        assert items.numel() == 0
