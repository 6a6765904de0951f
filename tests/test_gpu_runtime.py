"""The table runtime waits for one table's work only: the host-side calls
(status, info, download, free) of table A do not wait for a long sampling
run of table B on another stream, and freeing a table is stream-ordered."""
import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _long_sampling(tb, stream, out, rounds):
    """Enqueue `rounds` samplings of len(out) draws of table B on `stream`
    and return an event recorded after them."""
    done = torch.cuda.Event()
    with torch.cuda.stream(stream):
        for r in range(rounds):
            tb.sample(out.numel(), seed=100 + r, out=out, stream=stream)
        done.record(stream)
    return done


def test_status_of_one_table_does_not_wait_for_another_tables_sampling():
    wa = WL.f32_zipf(50_000, 1.0, 31)
    wb = WL.f32_uniform(10_000_000, 32)
    with wrs.AliasTable(len(wa)) as ta, wrs.AliasTable(len(wb)) as tb:
        ta.build(G.to_device(wa))
        tb.build(G.to_device(wb))
        assert ta.status() == wrs.OK and tb.status() == wrs.OK  # both built; the first waits warm up
        side = torch.cuda.Stream()
        out = torch.empty(1 << 29, dtype=torch.int32, device="cuda")  # 2 GB of samples per round
        done = _long_sampling(tb, side, out, rounds=8)  # about 0.1 s of device work
        assert ta.status() == wrs.OK
        info = ta.info()
        thr, alias, _ = ta.download()
        still_running = not done.query()
        side.synchronize()
        assert still_running, "table A's host calls waited for table B's sampling"
        qz, want = O.build_table(wa)
        assert info.Q == qz.Q
        assert np.array_equal(thr, want.thr) and np.array_equal(alias, want.alias)


def test_free_is_stream_ordered():
    w = WL.f32_zipf(3_000_000, 1.0, 33)
    qz, want = O.build_table(w)
    k = 1 << 28
    side = torch.cuda.Stream()
    out = torch.empty(k, dtype=torch.int32, device="cuda")
    t = wrs.AliasTable(len(w))
    t.build(G.to_device(w))
    assert t.status() == wrs.OK
    done = _long_sampling(t, side, out, rounds=4)
    t.free()  # returns at once; the memory goes back after the sampling
    still_running = not done.query()
    side.synchronize()
    assert still_running, "free waited for the sampling"
    idx = np.unique(np.random.default_rng(3).integers(0, k, size=20_000)).astype(np.uint64)
    got = out.cpu().numpy().view(np.uint32)[idx.astype(np.int64)]
    ref = O.sample_at(want.thr, want.alias, want.Qp, 103, 0, idx)
    assert np.array_equal(got, ref)
