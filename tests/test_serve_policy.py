"""Serving policy on the host (no GPU): the seeded request stream and the
resident-table cache (LRU order, pins, byte budget, pools)."""
import numpy as np

from paper_1903_00227_gb300 import serve as S


def test_request_stream_is_seeded_and_well_formed():
    a = S.request_stream(3000, rate=1000.0, seed=5)
    b = S.request_stream(3000, rate=1000.0, seed=5)
    assert [(r.arrival, r.table, r.k, r.build) for r in a] == [(r.arrival, r.table, r.k, r.build) for r in b]
    arr = np.array([r.arrival for r in a])
    assert (np.diff(arr) > 0).all()
    assert abs(len(a) / arr[-1] - 1000.0) < 100.0  # Poisson rate
    builds = [r for r in a if r.build]
    assert 0.25 < len(builds) / len(a) < 0.35
    assert all((1 << 10) <= r.n <= (1 << 24) for r in builds)
    assert all(1 <= r.k <= 10 ** 5 for r in a)
    seen = set()
    for r in a:
        if r.build:
            assert r.table not in seen  # a build request brings a new table
            seen.add(r.table)
        else:
            assert r.table in seen  # a sample-only request names a table built earlier
    assert len({r.stream_id for r in a}) == len(a)


def test_table_class_and_bytes():
    assert S.table_class(1) == 10 and S.table_class(1024) == 10 and S.table_class(1025) == 11
    assert S.table_class(1 << 24) == 24
    assert S.table_bytes(1 << 20) >= 16 << 20


class Obj:
    def __init__(self, cap):
        self.cap = cap


def test_cache_lru_pins_and_budget():
    one = S.table_bytes(1 << 10)
    c = S.TableCache(budget=3 * one)
    created, freed = [], []

    def create(cap):
        o = Obj(cap)
        created.append(o)
        return o

    for tid in range(3):
        o, cls = c.acquire(10, create, freed.append)
        assert cls == 10
        c.insert(tid, cls, o)
    assert len(created) == 3 and c.used == 3 * one
    c.get(0)  # 0 becomes most recent: LRU order 1, 2, 0
    c.pin(1)
    o, cls = c.acquire(10, create, freed.append)  # takes 2's object (1 is pinned)
    assert len(created) == 3 and 2 not in c.resident and c.evictions == 1
    c.insert(3, cls, o)
    c.pin(0)
    c.pin(3)
    assert c.acquire(10, create, freed.append) is None  # everything pinned, budget full
    c.unpin(0)
    assert c.acquire(10, create, freed.append) is not None  # 0's object now
    assert 0 not in c.resident and 1 in c.resident and 3 in c.resident and not freed


def test_cache_serves_small_tables_from_larger_pooled_objects():
    c = S.TableCache(budget=10 * S.table_bytes(1 << 14))
    assert c.reserve(14, Obj) and c.reserve(12, Obj)
    o, cls = c.acquire(11, Obj, None)  # smallest pooled class >= 11
    assert cls == 12 and o.cap == 1 << 12
    o, cls = c.acquire(11, Obj, None)
    assert cls == 14
    o, cls = c.acquire(11, Obj, None)  # pool empty: a new class-11 object within the budget
    assert cls == 11 and c.created == 3


def test_cache_frees_smaller_objects_for_a_large_table():
    small, big = S.table_bytes(1 << 10), S.table_bytes(1 << 12)
    c = S.TableCache(budget=2 * small + big - 1)
    freed = []
    for tid in range(2):
        o, cls = c.acquire(10, Obj, freed.append)
        c.insert(tid, cls, o)
    c.pin(1)
    c.pin(0)
    # no object of class >= 12 exists and both small tables are pinned
    assert c.acquire(12, Obj, freed.append) is None
    c.unpin(0)
    # the unpinned small table is freed (the pinned one stays) and a class-12 object fits
    o, cls = c.acquire(12, Obj, freed.append)
    assert cls == 12 and len(freed) == 1 and 0 not in c.resident and 1 in c.resident
    assert c.used <= c.budget and c.freed == 1


def test_summary_counts_per_run():
    """The summary of one run: latency percentiles, rates and the share of
    sample-only requests that found their table resident."""
    reqs = S.request_stream(1000, rate=1000.0, seed=9)
    n_sample_only = sum(1 for r in reqs if not r.build)
    lat = np.linspace(0.001, 0.1, len(reqs))
    res = {"latency": lat, "wall": 2.0, "ticks": 40, "evictions": 12, "rebuilds": n_sample_only // 4}
    s = S.summarize(res, reqs)
    assert s["requests"] == 1000 and s["requests_per_s"] == 500.0
    assert s["builds"] == len(reqs) - n_sample_only
    assert s["p50_ms"] == np.percentile(lat * 1e3, 50) and s["p99_ms"] == np.percentile(lat * 1e3, 99)
    assert s["evictions"] == 12 and s["rebuilds"] == n_sample_only // 4
    assert abs(s["sample_hit_rate"] - (1 - (n_sample_only // 4) / n_sample_only)) < 1e-12
    assert s["gsamples_s"] == sum(r.k for r in reqs) / 2.0 / 1e9
