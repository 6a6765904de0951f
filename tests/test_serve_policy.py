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
        o = c.acquire(10, create, freed.append)
        assert o is not None
        c.insert(tid, 10, o)
    assert len(created) == 3 and c.used == 3 * one
    c.get(0)  # 0 becomes most recent: LRU order 1, 2, 0
    c.pin(1)
    o = c.acquire(10, create, freed.append)  # evicts 2 (1 is pinned), reuses its object
    assert o is not None and len(created) == 3 and 2 not in c.resident and c.evictions == 1
    c.insert(3, 10, o)
    c.pin(0)
    c.pin(3)
    assert c.acquire(10, create, freed.append) is None  # everything pinned, budget full
    c.unpin(0)
    assert c.acquire(10, create, freed.append) is not None  # 0 evicted now
    assert 0 not in c.resident and 1 in c.resident and 3 in c.resident


def test_cache_frees_pooled_objects_of_other_classes():
    small, big = S.table_bytes(1 << 10), S.table_bytes(1 << 12)
    c = S.TableCache(budget=2 * small + big - 1)
    freed = []
    for tid in range(2):
        c.insert(tid, 10, c.acquire(10, Obj, freed.append))
    # a class-12 table does not fit: both class-10 tables are evicted into the
    # pool, then pooled objects are freed until it fits
    o = c.acquire(12, Obj, freed.append)
    assert o is not None and o.cap == 1 << 12
    assert len(freed) >= 1 and c.used <= c.budget
