"""Serving (continuous batching over resident tables) on the GPU: every
request's samples are the same served in a mix, on the plain one-request-at-
a-time path and from the CPU oracle, also when a small memory budget forces
evictions and rebuilds; and wrs_sample_many equals one wrs_sample per task."""
import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import serve as S
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs

pytestmark = pytest.mark.gpu

MASK64 = (1 << 64) - 1


def _requests(nreq, seed, rate=20000.0):
    return S.request_stream(nreq, rate=rate, seed=seed, n_lo=1 << 10, n_hi=1 << 16, k_hi=5000)


@pytest.fixture(scope="module")
def payload():
    return S.WeightSource(torch, max_class=16, variants=3)


def _oracle_samples(r, payload):
    w = payload.host(r.table, r.n).numpy().copy()
    _, tab = O.build_table(w)
    return O.sample(tab.thr, tab.alias, tab.Qp, r.k, r.seed & MASK64, r.stream_id)


def test_served_equals_plain_and_oracle(payload):
    reqs = _requests(400, 3)
    srv = S.Server(budget=2 << 30, max_inflight=3, tick_requests=64, tick_samples=1 << 20, payload=payload)
    assert srv.reserve(reqs, fill=0.1) > 0
    try:
        served = srv.run(reqs, keep_outputs=True)
        assert served["ticks"] > 3, "requests must be batched over several overlapping ticks"
        srv.cache.clear_resident()
        plain = srv.run_plain(reqs, keep_outputs=True)
        # every table fits the budget: nothing evicted, every sample-only request hits
        assert served["evictions"] == plain["evictions"] == 0
        assert served["rebuilds"] == plain["rebuilds"] == 0
    finally:
        srv.close()
    for r in reqs:
        assert np.array_equal(served["outputs"][r.rid], plain["outputs"][r.rid]), r
    for r in reqs[:25] + [r for r in reqs if not r.build][:15]:
        assert np.array_equal(served["outputs"][r.rid], _oracle_samples(r, payload)), r


def test_tiny_budget_evicts_and_rebuilds_same_results(payload):
    reqs = _requests(300, 8)
    small = S.Server(budget=6 * S.table_bytes(1 << 16), max_inflight=2, tick_requests=8, tick_samples=1 << 18,
                     payload=payload)
    big = S.Server(budget=2 << 30, max_inflight=1, tick_requests=1, tick_samples=1 << 18, payload=payload)
    try:
        a = small.run(reqs, keep_outputs=True)
        assert a["evictions"] > 10 and a["rebuilds"] > 0
        assert S.summarize(a, reqs)["sample_hit_rate"] < 1.0
        b = big.run(reqs, keep_outputs=True)
        assert b["evictions"] == 0 and b["rebuilds"] == 0
    finally:
        small.close()
        big.close()
    for r in reqs:
        assert np.array_equal(a["outputs"][r.rid], b["outputs"][r.rid]), r


def test_sample_many_equals_sample_per_task():
    wa = WL.f32_uniform(1000, 1)
    wb = WL.f32_zipf(70_000, 1.0, 2)
    with wrs.AliasTable(len(wa)) as A, wrs.AliasTable(len(wb)) as B:
        A.build(torch.from_numpy(wa).cuda())
        B.build(torch.from_numpy(wb).cuda())
        plan = [(A, len(wa), 10, 5, 0), (B, len(wb), 0, 6, 1), (B, len(wb), 5000, 7, 2),
                (A, len(wa), 3000, 8, 3), (B, len(wb), 1, 2 ** 63 + 9, 2 ** 40)]
        tasks = np.zeros((len(plan), 8), np.uint64)
        off = 0
        for i, (t, n, k, seed, sid) in enumerate(plan):
            tasks[i] = (wrs.table_buckets(t.handle), wrs.table_device_header(t.handle), n, k, seed, sid, off, 0)
            off += k
        d_tasks = torch.from_numpy(tasks.view(np.int64)).cuda()
        out = torch.full((off,), -1, dtype=torch.int32, device="cuda")
        assert wrs.sample_many(d_tasks.data_ptr(), len(plan), off, out.data_ptr(), 0) == wrs.OK
        got = out.cpu().numpy().view(np.uint32)
        o = 0
        for t, n, k, seed, sid in plan:
            if k:
                want = t.sample(k, seed, sid).cpu().numpy().view(np.uint32)
                assert np.array_equal(got[o:o + k], want)
            o += k
        assert wrs.sample_many(d_tasks.data_ptr(), 0, 5, out.data_ptr(), 0) == wrs.EINVAL
        assert wrs.sample_many(0, 0, 0, 0, 0) == wrs.OK  # nothing to draw
