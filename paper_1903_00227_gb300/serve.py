"""Continuous-batching request server over device-resident alias tables.

Serving is not in the paper (it builds one table and queries it); it is the
way a system uses the paper's two operations -- build(weights) -> table and
sample(table, k, seed) -> indices (Sec. 2.2) -- under a stream of requests.

A request either builds a table (its weights arrive with it) and samples it,
or samples a table that is already resident.  The server runs ticks:

* admission: every request that has arrived is admitted when a tick slot is
  free (at most ``max_inflight`` ticks on the GPU at once, at most
  ``tick_requests`` requests and ``tick_samples`` samples per tick) and the
  device-memory budget can hold the tables it needs; least-recently-used
  resident tables that no in-flight tick uses are evicted to make room;
* device work of a tick: for each build, the upload of its weights from
  pinned host memory and the build, on ``build_streams`` streams (table
  objects come from pools reserved at start-up: a table of n weights takes
  the smallest free object of capacity >= n, so the steady state allocates
  nothing), then ONE ``wrs_sample_many`` launch for all the tick's sample
  requests -- old and new tables alike -- and one device-to-host copy of the
  outputs; ticks overlap each other on the device;
* completion: a tick's requests complete when its copy has landed.

Every result is a pure function of (table weights, seed, stream id): a
request gets the same samples alone, in any mix, and on the plain path (one
request at a time: build if needed, ``wrs_sample``, copy, synchronise).

The policy pieces (``TableCache``, ``request_stream``) are plain Python and
hold no method arithmetic; the device work is the C ABI of libwrs.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import workloads as WL

TABLE_MIN_CAP = 1 << 10
BUCKET_BYTES = 16
WORKSPACE_BYTES_PER_TILE = 2 * 48 + 16 + 64 + 16  # tile sums, split, member list, chunk share


def table_class(n: int) -> int:
    """Capacity class of a table of n weights: capacity 2^c >= n, at least 2^10."""
    return max(10, int(math.ceil(math.log2(max(n, 1)))))


def table_bytes(cap: int) -> int:
    """Device bytes of a table of capacity cap (buckets + workspace, rounded up)."""
    tiles = (cap + 2047) // 2048
    return cap * BUCKET_BYTES + tiles * WORKSPACE_BYTES_PER_TILE + (64 << 10)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float      # seconds after the start of the run
    table: int          # table id
    n: int              # weights of the table
    k: int              # samples
    seed: int
    stream_id: int
    build: bool         # carries the table's weights (else: sample a resident table)


def request_stream(nreq: int, rate: float, seed: int, build_frac: float = 0.3, n_lo: int = 1 << 10,
                   n_hi: int = 1 << 24, k_lo: int = 1, k_hi: int = 10 ** 5, recent: int = 64):
    """Seeded request stream: Poisson arrivals at `rate` per second; a request
    builds a new table (Zipf 1.0 binary32 weights, size log-uniform in
    [n_lo, n_hi]) with probability build_frac, else samples one of the
    `recent` most recently built tables (the j-th most recent with weight
    1/(j+1)); k log-uniform in [k_lo, k_hi]."""
    u = (WL.words(4 * nreq, seed, 7) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    gaps = -np.log1p(-u[0::4]) / rate
    arrivals = np.cumsum(gaps)
    is_build = u[1::4] < build_frac
    sizes = WL.log_uniform_ints(nreq, n_lo, n_hi, seed, 8)
    ks = WL.log_uniform_ints(nreq, k_lo, k_hi, seed, 9)
    pick = u[2::4]
    built = []  # table ids, oldest first
    sizes_of = {}
    reqs = []
    for i in range(nreq):
        if is_build[i] or not built:
            tid = len(sizes_of)
            sizes_of[tid] = int(sizes[i])
            built.append(tid)
            reqs.append(Request(i, float(arrivals[i]), tid, sizes_of[tid], int(ks[i]), seed * 1000 + i, i, True))
        else:
            m = min(recent, len(built))
            wts = 1.0 / np.arange(1, m + 1)
            j = int(np.searchsorted(np.cumsum(wts) / wts.sum(), pick[i], side="right"))
            tid = built[-1 - min(j, m - 1)]
            reqs.append(Request(i, float(arrivals[i]), tid, sizes_of[tid], int(ks[i]), seed * 1000 + i, i, False))
    return reqs


MAX_CLASS = 32


class TableCache:
    """Resident tables in LRU order under a byte budget.  A table used by an
    in-flight tick is pinned and never evicted.  Table objects live on after
    eviction in pools by capacity class (2^c); pooled objects count against
    the budget too.  A table of class c takes the smallest pooled object of
    class >= c; else a new object if the budget allows; else the object of
    the least recently used unpinned table of class >= c; else pooled and
    unpinned resident objects of smaller classes are freed until a new one
    fits."""

    def __init__(self, budget: int):
        self.budget = budget
        self.resident = collections.OrderedDict()  # table id -> (cls of the object, obj)
        self.pins = collections.Counter()
        self.pool = collections.defaultdict(list)  # cls -> [obj]
        self.used = 0  # bytes of resident + pooled objects
        self.evictions = 0
        self.created = 0
        self.freed = 0

    def get(self, tid):
        e = self.resident.get(tid)
        if e is not None:
            self.resident.move_to_end(tid)
        return e

    def pin(self, tid):
        self.pins[tid] += 1

    def unpin(self, tid):
        self.pins[tid] -= 1
        if self.pins[tid] <= 0:
            del self.pins[tid]

    def reserve(self, cls: int, create) -> bool:
        """Create one pooled object of class cls if the budget allows."""
        need = table_bytes(1 << cls)
        if self.used + need > self.budget:
            return False
        self.used += need
        self.created += 1
        self.pool[cls].append(create(1 << cls))
        return True

    def acquire(self, cls: int, create, free):
        """(object, its class) for a new resident table of class cls, or None
        when nothing can be had until in-flight ticks complete."""
        for c in range(cls, MAX_CLASS + 1):
            if self.pool.get(c):
                return self.pool[c].pop(), c
        need = table_bytes(1 << cls)
        if self.used + need <= self.budget:
            self.used += need
            self.created += 1
            return create(1 << cls), cls
        for tid, (c, obj) in self.resident.items():  # least recently used first
            if c >= cls and tid not in self.pins:
                del self.resident[tid]
                self.evictions += 1
                return obj, c
        # make room from smaller objects: pooled first, then unpinned residents (LRU)
        smaller = [(c, o) for c in sorted(self.pool) if c < cls for o in self.pool[c]]
        smaller += [(c, o, tid) for tid, (c, o) in self.resident.items() if c < cls and tid not in self.pins]
        room = self.budget - self.used + sum(table_bytes(1 << e[0]) for e in smaller)
        if room < need:
            return None
        for e in smaller:
            if self.used + need <= self.budget:
                break
            c, o = e[0], e[1]
            if len(e) == 3:
                del self.resident[e[2]]
                self.evictions += 1
            else:
                self.pool[c].remove(o)
            free(o)
            self.freed += 1
            self.used -= table_bytes(1 << c)
        self.used += need
        self.created += 1
        return create(1 << cls), cls

    def insert(self, tid, cls, obj):
        self.resident[tid] = (cls, obj)

    def clear_resident(self):
        """Return every resident table's object to the pool (between runs)."""
        for tid, (cls, obj) in list(self.resident.items()):
            self.pool[cls].append(obj)
        self.resident.clear()


class WeightSource:
    """Request payloads: the weights of table t are the first n entries of one
    of `variants` binary32 Zipf(1.0) arrays of 2^max_class weights (randomly
    permuted ranks, workloads.f32_zipf's recipe made on the device), kept in
    pinned host memory; a build uploads them like a client's payload."""

    def __init__(self, torch, max_class: int = 24, variants: int = 4):
        self.max_n = 1 << max_class
        self.arrays = []
        for v in range(variants):
            d = WL.generate_device("f32_zipf", self.max_n, 0x5EED + v, 1.0)
            h = torch.empty(self.max_n, dtype=torch.float32, pin_memory=True)
            h.copy_(d)
            self.arrays.append(h)
        torch.cuda.synchronize()

    def host(self, table: int, n: int):
        """Pinned host tensor view of table `table`'s n weights."""
        if n > self.max_n:
            raise ValueError("table larger than the payload source")
        return self.arrays[table % len(self.arrays)][:n]


# ------------------------------------------------------------------ GPU side
class _Slot:
    """Pinned host and device buffers of one in-flight tick."""

    def __init__(self, torch, max_tasks: int, max_samples: int):
        self.h_tasks = torch.zeros((max_tasks, 8), dtype=torch.int64, pin_memory=True)
        self.d_tasks = torch.zeros((max_tasks, 8), dtype=torch.int64, device="cuda")
        self.d_out = torch.empty(max_samples, dtype=torch.int32, device="cuda")
        self.h_out = torch.empty(max_samples, dtype=torch.int32, pin_memory=True)
        self.done = None
        self.reqs = []
        self.tables = []
        self.keep = []
        self.total_k = 0


class Server:
    """Continuous-batching server (see module docstring) on the current GPU."""

    def __init__(self, budget: int = 40 << 30, max_inflight: int = 3, tick_requests: int = 2048,
                 tick_samples: int = 1 << 24, build_streams: int = 4, payload: "WeightSource | None" = None):
        import torch

        from . import wrs

        self.torch, self.wrs = torch, wrs
        self.payload = payload or WeightSource(torch)
        self.cache = TableCache(budget)
        self.max_inflight = max_inflight
        self.tick_requests = tick_requests
        self.tick_samples = tick_samples
        self.bstreams = [torch.cuda.Stream() for _ in range(build_streams)]
        self.sstream = torch.cuda.Stream()
        self.slots = [_Slot(torch, tick_requests, tick_samples) for _ in range(max_inflight)]
        self.last_use = {}  # id(table object) -> event of the last tick that read it
        self.ptrs = {}      # id(table object) -> (buckets, header)
        self.rebuilds = 0   # sample-only requests of the current run whose table had been evicted

    # -- table objects
    def _create(self, cap):
        t = self.wrs.AliasTable(cap)
        self.ptrs[id(t)] = (self.wrs.table_buckets(t.handle), self.wrs.table_device_header(t.handle))
        return t

    def _free(self, t):
        self.ptrs.pop(id(t), None)
        self.last_use.pop(id(t), None)
        t.free()

    def reserve(self, reqs, fill: float = 0.9) -> int:
        """Start-up: pool table objects for the size classes that `reqs` build,
        in proportion to how often each class is built, filling `fill` of the
        budget.  Returns the number of objects created."""
        counts = collections.Counter(table_class(r.n) for r in reqs if r.build)
        if not counts:
            return 0
        total = sum(counts.values())
        unit = sum(m / total * table_bytes(1 << c) for c, m in counts.items())
        units = fill * self.cache.budget / unit
        made = 0
        for c, m in sorted(counts.items()):
            for _ in range(max(1, int(m / total * units))):
                if not self.cache.reserve(c, self._create):
                    break
                made += 1
        self.torch.cuda.synchronize()
        return made

    def _build(self, req, stream):
        """Upload req's table weights (its payload) on `stream` and build the
        table there; returns (table object, staging buffer) or None when no
        table object can be had now."""
        r = self.cache.acquire(table_class(req.n), self._create, self._free)
        if r is None:
            return None
        t, cls = r
        ev = self.last_use.get(id(t))
        if ev is not None:
            stream.wait_event(ev)
        with self.torch.cuda.stream(stream):
            w = self.torch.empty(req.n, dtype=self.torch.float32, device="cuda")
            w.copy_(self.payload.host(req.table, req.n), non_blocking=True)
            t.build(w, stream=stream.cuda_stream)
        self.cache.insert(req.table, cls, t)
        return t, w

    def close(self):
        self.torch.cuda.synchronize()
        for cls, objs in self.cache.pool.items():
            for t in objs:
                self._free(t)
        for tid, (cls, t) in self.cache.resident.items():
            self._free(t)
        self.cache = TableCache(self.cache.budget)

    # -- continuous batching
    def run(self, reqs, keep_outputs: bool = False):
        if any(r.k > self.tick_samples for r in reqs):
            raise ValueError("a request draws more samples than one tick holds")
        """Serve `reqs` (sorted by arrival) against the wall clock; returns
        per-request latency in seconds, completion order checksums and, when
        asked, each request's samples."""
        torch, wrs = self.torch, self.wrs
        N = len(reqs)
        lat = np.zeros(N)
        sums = np.zeros(N, dtype=np.uint64)
        outs = [None] * N if keep_outputs else None
        free_slots = list(self.slots)
        inflight = collections.deque()
        nxt = 0
        pending = collections.deque()  # arrived, not yet admitted
        ev0, self.rebuilds = self.cache.evictions, 0
        t0 = time.perf_counter()
        ticks = 0

        def finish(slot, now):
            h = slot.h_out[:slot.total_k].numpy().view(np.uint32)
            for req, off in slot.reqs:
                seg = h[off:off + req.k]
                lat[req.rid] = now - req.arrival
                sums[req.rid] = np.uint64(int(seg.astype(np.uint64).sum()) & 0xFFFFFFFFFFFFFFFF)
                if outs is not None:
                    outs[req.rid] = seg.copy()
            for tid in slot.tables:
                self.cache.unpin(tid)
            slot.reqs, slot.tables, slot.keep = [], [], []
            free_slots.append(slot)

        while nxt < N or pending or inflight:
            now = time.perf_counter() - t0
            while inflight and inflight[0].done.query():
                finish(inflight.popleft(), time.perf_counter() - t0)
            while nxt < N and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            if pending and free_slots:
                slot = free_slots.pop()
                self._issue(slot, pending)
                if slot.reqs:
                    inflight.append(slot)
                    ticks += 1
                else:
                    free_slots.append(slot)
                    if not inflight:
                        raise RuntimeError("request cannot be admitted: budget or tick limits too small")
                    inflight[0].done.synchronize()
                continue
            if inflight:
                if not pending and nxt < N and reqs[nxt].arrival > now:
                    time.sleep(0)
                continue
            if nxt < N:
                delay = reqs[nxt].arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(min(delay, 0.001))
        wall = time.perf_counter() - t0
        return {"latency": lat, "checksum": sums, "outputs": outs, "wall": wall, "ticks": ticks,
                "evictions": self.cache.evictions - ev0, "rebuilds": self.rebuilds}

    def _issue(self, slot, pending):
        """Admit pending requests into `slot` and launch its device work."""
        torch, wrs = self.torch, self.wrs
        tasks = slot.h_tasks.numpy().view(np.uint64)
        off = 0
        nb = 0
        build_events = []
        while pending and len(slot.reqs) < self.tick_requests:
            req = pending[0]
            if off + req.k > self.tick_samples:
                break
            e = self.cache.get(req.table)
            if e is None:  # a build, or a sample of an evicted table: (re)build it
                stream = self.bstreams[nb % len(self.bstreams)]
                r = self._build(req, stream)
                if r is None:
                    break  # no memory until in-flight ticks complete
                t, w = r
                if not req.build:
                    self.rebuilds += 1
                slot.keep.append(w)
                ev = torch.cuda.Event()
                ev.record(stream)
                build_events.append(ev)
                nb += 1
            else:
                t = e[1]
            pending.popleft()
            self.cache.pin(req.table)
            slot.tables.append(req.table)
            bp, hp = self.ptrs[id(t)]
            i = len(slot.reqs)
            tasks[i] = (bp, hp, req.n, req.k, req.seed & 0xFFFFFFFFFFFFFFFF, req.stream_id, off, 0)
            slot.reqs.append((req, off))
            slot.keep.append(t)
            off += req.k
        if not slot.reqs:
            return
        nt = len(slot.reqs)
        slot.total_k = off
        s = self.sstream
        for ev in build_events:
            s.wait_event(ev)
        with torch.cuda.stream(s):
            slot.d_tasks[:nt].copy_(slot.h_tasks[:nt], non_blocking=True)
            if off:
                rc = wrs.sample_many(slot.d_tasks.data_ptr(), nt, off, slot.d_out.data_ptr(), s.cuda_stream)
                if rc != wrs.OK:
                    raise wrs.WrsError(rc, "wrs_sample_many")
                slot.h_out[:off].copy_(slot.d_out[:off], non_blocking=True)
            done = torch.cuda.Event()
            done.record(s)
        slot.done = done
        for t in slot.keep:
            if hasattr(t, "handle"):
                self.last_use[id(t)] = done

    # -- the plain path: one request at a time
    def run_plain(self, reqs, keep_outputs: bool = False):
        torch, wrs = self.torch, self.wrs
        N = len(reqs)
        lat = np.zeros(N)
        sums = np.zeros(N, dtype=np.uint64)
        outs = [None] * N if keep_outputs else None
        slot = self.slots[0]
        s = self.sstream
        ev0, rebuilds = self.cache.evictions, 0
        t0 = time.perf_counter()
        for req in reqs:
            delay = req.arrival - (time.perf_counter() - t0)
            while delay > 0:
                time.sleep(min(delay, 0.001))
                delay = req.arrival - (time.perf_counter() - t0)
            e = self.cache.get(req.table)
            if e is None:
                r = self._build(req, s)
                if r is None:
                    raise RuntimeError("budget too small for one table")
                t = r[0]
                rebuilds += 0 if req.build else 1
            else:
                t = e[1]
            with torch.cuda.stream(s):
                if req.k:
                    t.sample(req.k, req.seed & 0xFFFFFFFFFFFFFFFF, req.stream_id, out=slot.d_out,
                             stream=s.cuda_stream)
                    slot.h_out[:req.k].copy_(slot.d_out[:req.k], non_blocking=True)
            s.synchronize()
            seg = slot.h_out[:req.k].numpy().view(np.uint32)
            lat[req.rid] = time.perf_counter() - t0 - req.arrival
            sums[req.rid] = np.uint64(int(seg.astype(np.uint64).sum()) & 0xFFFFFFFFFFFFFFFF)
            if outs is not None:
                outs[req.rid] = seg.copy()
        wall = time.perf_counter() - t0
        return {"latency": lat, "checksum": sums, "outputs": outs, "wall": wall, "ticks": N,
                "evictions": self.cache.evictions - ev0, "rebuilds": rebuilds}


def summarize(res, reqs) -> dict:
    lat = res["latency"] * 1e3
    n_build = sum(1 for r in reqs if r.build)
    n_sample_only = len(reqs) - n_build
    return {"requests": len(reqs), "wall_s": res["wall"], "requests_per_s": len(reqs) / res["wall"],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "builds": n_build,
            "gsamples_s": sum(r.k for r in reqs) / res["wall"] / 1e9,
            "gweights_built_s": sum(r.n for r in reqs if r.build) / res["wall"] / 1e9,
            "ticks": res["ticks"], "evictions": res["evictions"], "rebuilds": res["rebuilds"],
            "sample_hit_rate": 1.0 - res["rebuilds"] / max(n_sample_only, 1)}
