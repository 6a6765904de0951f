"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tables must be identical bucket for bucket (thresholds and aliases) to the
oracle's Alg. 2 table, the header (Q, beta, shift, qp, light count) must match
the oracle's exact units, and samples must be identical index for index to
the oracle's queries (integer work: bit-exact).  Sizes span several 2048-item
tiles with ragged tails; inputs include the paper's workload shapes
(uniform, Zipf-permuted) and degenerate ones.
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
SCAN_CHUNK = 256 * TILE


def _inputs():
    rng = np.random.default_rng(123)
    cases = []
    for n in (1, 2, 3, 17, TILE - 1, TILE, TILE + 1, 2 * TILE + 5, 3 * TILE + 17, 100_003):
        cases.append((f"u32_uniform_{n}", WL.u32_uniform(n, n)))
        cases.append((f"f32_uniform_{n}", WL.f32_uniform(n, n + 1)))
        cases.append((f"zipf1_{n}", WL.f32_zipf(n, 1.0, n + 2)))
    for s in (0.5, 0.8, 1.5, 2.0, 3.0):
        cases.append((f"zipf{s}_60000", WL.f32_zipf(60_000, s, 7)))
    n = 50_000
    base = WL.u32_uniform(n, 9)
    cases.append(("sorted_asc", np.sort(base)))
    cases.append(("sorted_desc", np.sort(base)[::-1].copy()))
    cases.append(("all_equal", np.full(n, 77, np.uint32)))
    cases.append(("all_equal_f32", np.full(n, 0.1, np.float32)))
    g = np.ones(n, np.uint32)
    g[n // 3] = 10_000_000
    cases.append(("one_giant", g))
    cases.append(("small_ints_with_zeros", rng.integers(0, 4, n).astype(np.uint32)))
    z = np.zeros(n, np.uint32)
    z[::97] = 5
    cases.append(("mostly_zero", z))
    tv = np.where(rng.random(n) < 0.1, 9, 1).astype(np.uint32)
    cases.append(("two_values", tv))
    wide = (rng.random(n) * np.exp2(rng.integers(-30, 20, n))).astype(np.float32)
    cases.append(("f32_wide_range", wide))
    sub = (rng.integers(1, 1 << 23, n) * 2.0 ** -149).astype(np.float32)
    cases.append(("f32_subnormal", sub))
    heavy_first = np.concatenate([np.full(n // 10, 1000, np.uint32), np.ones(n - n // 10, np.uint32)])
    cases.append(("heavies_first", heavy_first))
    cases.append(("heavies_last", heavy_first[::-1].copy()))
    return cases


CASES = _inputs()


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_table_and_samples_match_oracle(name, w):
    qz, tab = O.build_table(w)
    n = len(w)
    with G.gpu_build(w) as t:
        assert t.status() == wrs.OK
        info = t.info()
        assert info.Q == qz.Q and info.beta == qz.beta
        assert info.shift == tab.shift and info.qp == tab.Qp
        n_light = sum(1 for i in range(n) if n * qz.q_int(i) <= qz.Q) if n < 5000 else None
        if n_light is not None:
            assert info.n_light == n_light
        thr, alias, res = t.download()
        bad = np.nonzero((thr != tab.thr) | (alias != tab.alias))[0]
        assert bad.size == 0, f"{bad.size} buckets differ, first {bad[:5]}: gpu {thr[bad[:3]]},{alias[bad[:3]]} oracle {tab.thr[bad[:3]]},{tab.alias[bad[:3]]}"
        assert not res.any()
        k = 3 * n + 7
        got = G.gpu_samples(t, k, seed=1000 + n, stream_id=5)
        want = O.sample(tab.thr, tab.alias, tab.Qp, k, 1000 + n, 5)
        assert np.array_equal(got, want)


def test_config1_exact_workload():
    """n = 10^6 uint32 weights uniform in [1, 2^24] from seed 1, then 10^6
    samples with seed 2: table and indices bit-exact."""
    w = WL.u32_uniform(1_000_000, 1)
    qz, tab = O.build_table(w)
    with G.gpu_build(w) as t:
        thr, alias, _ = t.download()
        assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias)
        got = G.gpu_samples(t, 1_000_000, seed=2)
    assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, 1_000_000, 2, 0))


def test_rebuild_same_table_object():
    with wrs.AliasTable(3 * TILE) as t:
        for seed, n in ((1, 3 * TILE), (2, 1000), (3, 2 * TILE + 1)):
            w = WL.f32_zipf(n, 1.0, seed)
            qz, tab = O.build_table(w)
            t.build(G.to_device(w))
            thr, alias, _ = t.download()
            assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias)


def test_sampler_alone_on_uploaded_oracle_table():
    w = WL.f32_zipf(30_000, 1.2, 5)
    qz, tab = O.build_table(w)
    n = len(w)
    buckets = np.zeros((n, 2), np.uint64)
    buckets[:, 0] = tab.thr
    buckets[:, 1] = tab.alias.astype(np.uint64)
    with wrs.AliasTable(n) as t:
        rc = wrs.table_upload(t.handle, buckets.ctypes.data, n, int(qz.Qw[0]), int(qz.Qw[1]), qz.beta)
        assert rc == wrs.OK
        t.n = n
        for seed, sid in ((0, 0), (7, 1), (2 ** 63 + 5, 2 ** 40 + 3)):
            got = G.gpu_samples(t, 123_457, seed, sid)
            assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, 123_457, seed, sid))


@pytest.mark.parametrize("bad,code", [(np.nan, wrs.EINVAL), (np.inf, wrs.EINVAL), (-1.0, wrs.EINVAL),
                                      (-0.0, wrs.EINVAL)])
def test_invalid_weights_reported(bad, code):
    w = WL.f32_uniform(10_000, 3)
    w[7777] = bad
    with G.gpu_build(w) as t:
        # sampling before the status is read: the kernel writes nothing
        out = torch.full((100,), -7, dtype=torch.int32, device="cuda")
        t.sample(100, 1, out=out)
        torch.cuda.synchronize()
        assert (out == -7).all(), "a failed table must not be sampled"
        assert t.status() == code
        # once the host has read the failure, the call returns it
        with pytest.raises(wrs.WrsError) as e:
            t.sample(100, 1, out=out)
        assert e.value.code == code


def test_all_zero_and_overflow_reported():
    with G.gpu_build(np.zeros(5000, np.float32)) as t:
        assert t.status() == wrs.EINVAL
    w = np.ones(5000, np.float32)
    w[0] = np.float32(2.0 ** -149)
    w[1] = np.float32(2.0 ** 100)
    with G.gpu_build(w) as t:
        assert t.status() == wrs.EOVERFLOW
    # every item fits in 95 bits, the total does not: q = 1 (x 4998), 2^94, 2^94
    w = np.full(5000, 2.0 ** -10, np.float32)
    w[1] = w[4000] = np.float32(2.0 ** 84)
    with G.gpu_build(w) as t:
        assert t.status() == wrs.EOVERFLOW
    w[4000] = np.float32(2.0 ** -10)  # Q = 2^94 + 4999 < 2^95: a valid table
    with G.gpu_build(w) as t:
        assert t.status() == wrs.OK and t.info().Q == 2 ** 94 + 4999


def test_bounded_wait_times_out_and_context_survives():
    """A tile that never publishes its look-back flag makes its successor's
    bounded wait run out: the build reports WRS_ETIMEOUT instead of hanging,
    and the same table then builds correctly."""
    w = WL.u32_uniform(5 * SCAN_CHUNK + 17, 4)
    with wrs.AliasTable(len(w)) as t:
        old = wrs.set_wait_limit(2000)
        try:
            wrs.debug_skip_publish(2)
            t.build(G.to_device(w))
            assert t.status() == wrs.ETIMEOUT
        finally:
            wrs.set_wait_limit(old)
            wrs.debug_skip_publish(-1)
        t.build(G.to_device(w))
        assert t.status() == wrs.OK
        qz, tab = O.build_table(w)
        thr, alias, _ = t.download()
        assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias)


def test_unaligned_weight_pointer():
    w = WL.f32_zipf(3 * TILE + 3, 1.0, 11)
    big = torch.from_numpy(np.concatenate([np.zeros(1, np.float32), w])).cuda()
    view = big[1:]
    assert view.data_ptr() % 16 != 0
    qz, tab = O.build_table(w)
    with wrs.AliasTable(len(w)) as t:
        t.build(view)
        thr, alias, _ = t.download()
    assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias)


def test_concurrent_tables_on_separate_streams():
    """Four table objects built and sampled on four CUDA streams with nothing
    ordering one stream against another: table objects share no state, so
    each table and its samples equal the oracle's for its own weights."""
    ws = [WL.f32_zipf(3 * TILE + 7 + 1001 * i, 1.0 + 0.25 * i, 40 + i) for i in range(3)]
    ws.append(WL.u32_uniform(5 * TILE + 3, 44))
    k = 100_003
    dev = [G.to_device(w) for w in ws]
    outs = [torch.empty(k, dtype=torch.int32, device="cuda") for _ in ws]
    streams = [torch.cuda.Stream() for _ in ws]
    tables = [wrs.AliasTable(len(w)) for w in ws]
    torch.cuda.synchronize()
    try:
        for t, d, st in zip(tables, dev, streams):
            t.build(d, stream=st)
        for i, (t, st) in enumerate(zip(tables, streams)):
            t.sample(k, 70 + i, i, out=outs[i], stream=st)
        torch.cuda.synchronize()
        for i, (w, t) in enumerate(zip(ws, tables)):
            qz, tab = O.build_table(w)
            assert t.status() == wrs.OK
            thr, alias, _ = t.download()
            assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias), i
            got = outs[i].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, k, 70 + i, i)), i
    finally:
        for t in tables:
            t.free()


def test_host_buffer_entry_points():
    w = WL.f32_uniform(20_000, 8)
    qz, tab = O.build_table(w)
    with wrs.AliasTable(len(w)) as t:
        assert wrs.table_build_host(t.handle, w.ctypes.data, len(w), wrs.F32, 0) == wrs.OK
        t.n = len(w)
        out = np.zeros(50_000, np.uint32)
        assert wrs.sample_host(t.handle, 50_000, 9, 1, out.ctypes.data, 0) == wrs.OK
    assert np.array_equal(out, O.sample(tab.thr, tab.alias, tab.Qp, 50_000, 9, 1))


def test_host_entry_points_double_buffered():
    """The end-to-end schedule the benchmark times: two table objects on two
    CUDA streams, step i+1's wrs_table_build_host issued before step i's
    wrs_sample_host, so an upload and a build overlap the other table's
    sampling.  Every step's samples equal the oracle's for its weights."""
    n, k = 3 * TILE + 11, 40_000
    inputs = [WL.f32_zipf(n, 1.0, 21), WL.f32_uniform(n, 22), WL.u32_uniform(n, 23).view(np.float32),
              WL.f32_zipf(n, 1.5, 24)]
    dtypes = [wrs.F32, wrs.F32, wrs.U32, wrs.F32]
    want = []
    for i, (w, dt) in enumerate(zip(inputs, dtypes)):
        qz, tab = O.build_table(w.view(np.uint32) if dt == wrs.U32 else w)
        want.append(O.sample(tab.thr, tab.alias, tab.Qp, k, 300 + i, 0))
    h_in = [torch.from_numpy(np.ascontiguousarray(w)).pin_memory() for w in inputs]
    h_out = [torch.empty(k, dtype=torch.int32).pin_memory() for _ in range(2)]
    tables = [wrs.AliasTable(n), wrs.AliasTable(n)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    try:
        def build(i):
            t = i % 2
            assert wrs.table_build_host(tables[t].handle, h_in[i].data_ptr(), n, dtypes[i],
                                        streams[t].cuda_stream) == wrs.OK
            tables[t].n = n

        build(0)
        for i in range(len(inputs)):
            if i + 1 < len(inputs):
                build(i + 1)
            t = i % 2
            assert wrs.sample_host(tables[t].handle, k, 300 + i, 0, h_out[t].data_ptr(),
                                   streams[t].cuda_stream) == wrs.OK
            got = h_out[t].numpy().view(np.uint32).copy()
            assert np.array_equal(got, want[i]), i
        torch.cuda.synchronize()
        assert all(t.status() == wrs.OK for t in tables)
    finally:
        for t in tables:
            t.free()


def test_build_options_do_not_change_the_table():
    """Alg. 3's table is Alg. 2's for every split count (reading 2): the
    first configuration's 64 splits, one split, a few, one per tile, and the
    128-bit walk forced, all give the oracle's table; accumulator mode U64
    fails only when Q >= 2^64."""
    cases = [WL.u32_uniform(1_000_000, 1), WL.f32_zipf(300_001, 1.5, 8), WL.f32_uniform(70_000, 9)]
    for w in cases:
        qz, tab = O.build_table(w)
        ntiles = -(-len(w) // 2048)
        w_dev = G.to_device(w)
        with wrs.AliasTable(len(w)) as t:
            for splits in sorted({0, 1, 2, 3, 64, ntiles} & set(range(ntiles + 1))):
                for acc in (wrs.ACC_AUTO, wrs.ACC_U128):
                    t.build_opts(w_dev, splits=splits, acc=acc, tile=2048 if splits == 1 else 0,
                                 window=2048 if splits == 2 else 0)
                    assert t.status() == wrs.OK, (splits, acc)
                    thr, alias, _ = t.download()
                    assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias), (len(w), splits, acc)
            t.build_opts(w_dev, acc=wrs.ACC_U64)
            assert t.status() == (wrs.OK if qz.Q < 1 << 64 else wrs.EOVERFLOW)
            got = G.gpu_samples(t.build(w_dev), 5000, seed=3) if qz.Q >= 1 << 64 else None
        if got is not None:  # a failed build does not stick: the next plain build is whole
            assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, 5000, 3, 0))
    with wrs.AliasTable(10) as t:
        w_dev = G.to_device(np.ones(10, np.uint32))
        for bad in (wrs.BuildOpts(splits=2), wrs.BuildOpts(tile=1024), wrs.BuildOpts(window=4096),
                    wrs.BuildOpts(acc=3), wrs.BuildOpts(flags=1)):
            assert wrs.table_build_opts(t.handle, w_dev.data_ptr(), 10, wrs.U32, bad, 0) == wrs.EINVAL
