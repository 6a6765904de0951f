"""Batched build and sampling (wrs_batch_*) vs the CPU oracle, table by table.

Every table of a batch must get exactly the oracle's Alg. 2 table for its
weights and exactly the oracle's samples for stream id stream_id + t, whatever
its neighbours are: sizes from 1 weight to many tiles with ragged tails,
binary32 and uint32 words, a failed table among good ones, replays of a
captured CUDA graph, and every sweep grouping the autotuner may pick.
"""
import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs

pytestmark = pytest.mark.gpu

TILE = 2048
SIZES = [1, 2, 3, 31, 32, 2047, 2048, 2049, 4101, 9000, 3 * TILE + 17, 70_001, 150_000, 5, 600_013]


def _weights(sizes, dtype, seed):
    out = []
    for t, n in enumerate(sizes):
        if dtype == "u32":
            out.append(WL.u32_uniform(n, seed + t))
        elif t % 2:
            out.append(WL.f32_zipf(n, 1.0 if t % 4 == 1 else 1.5, seed + t))
        else:
            out.append(WL.f32_uniform(n, seed + t))
    return out


def _to_cuda(ws):
    if ws[0].dtype == np.uint32:
        return [torch.from_numpy(w.view(np.int32).copy()).cuda() for w in ws]
    return [torch.from_numpy(w.copy()).cuda() for w in ws]


def _check_tables(b, ws):
    thr, alias, res = b.download()
    assert not res.any()
    for t, w in enumerate(ws):
        qz, tab = O.build_table(w)
        lo, hi = b.offsets[t], b.offsets[t] + len(w)
        assert np.array_equal(thr[lo:hi], tab.thr), f"table {t} thresholds"
        assert np.array_equal(alias[lo:hi], tab.alias), f"table {t} aliases"
        info = b.info(t)
        assert info.status == wrs.OK and info.Q == qz.Q and info.beta == qz.beta and info.qp == tab.Qp


def _check_samples(b, ws, ks, out, seed, sid):
    got = out.cpu().numpy().view(np.uint32)
    for t, w in enumerate(ws):
        _, tab = O.build_table(w)
        lo = b.k_offsets[t]
        want = O.sample(tab.thr, tab.alias, tab.Qp, ks[t], seed, sid + t)
        assert np.array_equal(got[lo:lo + ks[t]], want), f"table {t} samples"


@pytest.mark.parametrize("dtype", ["f32", "u32"])
def test_batch_matches_oracle_per_table(dtype):
    ws = _weights(SIZES, dtype, 40)
    with wrs.AliasBatch(SIZES) as b:
        buf = b.pack(_to_cuda(ws))
        b.build(buf)
        rc, st = b.status()
        assert rc == wrs.OK and st == [wrs.OK] * len(SIZES)
        _check_tables(b, ws)
        ks = [0 if t == 3 else (t * 997 + 1) for t in range(len(SIZES))]
        b.set_samples(ks)
        out = b.sample(seed=77, stream_id=1000)
        torch.cuda.synchronize()
        _check_samples(b, ws, ks, out, 77, 1000)


def test_batch_equals_single_table_path():
    ws = _weights(SIZES[:9], "f32", 3)
    with wrs.AliasBatch(SIZES[:9]) as b:
        b.build(b.pack(_to_cuda(ws)))
        thr, alias, _ = b.download()
        ks = [1000] * 9
        b.set_samples(ks)
        out = b.sample(seed=5, stream_id=9).cpu().numpy().view(np.uint32)
        for t, w in enumerate(ws):
            with wrs.AliasTable(len(w)) as a:
                a.build(torch.from_numpy(w).cuda())
                s_thr, s_alias, _ = a.download()
                single = a.sample(1000, 5, 9 + t).cpu().numpy().view(np.uint32)
            lo = b.offsets[t]
            assert np.array_equal(thr[lo:lo + len(w)], s_thr) and np.array_equal(alias[lo:lo + len(w)], s_alias)
            assert np.array_equal(out[b.k_offsets[t]:b.k_offsets[t] + 1000], single)


def test_failed_table_is_isolated():
    sizes = [5000, 3000, 7000, 100]
    ws = _weights(sizes, "f32", 11)
    ws[1] = ws[1].copy()
    ws[1][1234] = np.nan
    with wrs.AliasBatch(sizes) as b:
        b.build(b.pack(_to_cuda(ws)))
        rc, st = b.status()
        assert rc == wrs.EINVAL and st == [wrs.OK, wrs.EINVAL, wrs.OK, wrs.OK]
        ks = [500, 500, 500, 500]
        b.set_samples(ks)
        out = torch.full((2000,), -7, dtype=torch.int32, device="cuda")
        b.sample(3, 0, out=out)
        torch.cuda.synchronize()
        assert (out[500:1000] == -7).all(), "a failed table must not be sampled"
        thr, alias, _ = b.download()
        good = [0, 2, 3]
        got = out.cpu().numpy().view(np.uint32)
        for t in good:
            _, tab = O.build_table(ws[t])
            lo = b.offsets[t]
            assert np.array_equal(thr[lo:lo + sizes[t]], tab.thr) and np.array_equal(alias[lo:lo + sizes[t]], tab.alias)
            want = O.sample(tab.thr, tab.alias, tab.Qp, 500, 3, t)
            assert np.array_equal(got[b.k_offsets[t]:b.k_offsets[t] + 500], want)


def test_graph_capture_and_replay():
    """Build + sample captured once; replays after rewriting the weights in
    place give the oracle's tables and samples of the new weights (the
    look-back generation advances on the device)."""
    sizes = [3000, 1, 9000, 2 * TILE, 300_000]
    ks = [100, 5, 1000, 0, 4096]
    with wrs.AliasBatch(sizes) as b:
        ws0 = _weights(sizes, "f32", 100)
        buf = b.pack(_to_cuda(ws0))
        b.set_samples(ks)
        out = torch.empty(b.k_offsets[-1], dtype=torch.int32, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            b.build(buf)
            b.sample(21, 4, out=out)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.build(buf)
            b.sample(21, 4, out=out)
        for rep, seed in enumerate((200, 300, 200)):
            ws = _weights(sizes, "f32", seed)
            buf.copy_(b.pack(_to_cuda(ws)))
            g.replay()
            torch.cuda.synchronize()
            rc, st = b.status()
            assert rc == wrs.OK, (rep, st)
            _check_tables(b, ws)
            _check_samples(b, ws, ks, out, 21, 4)


def test_tuner_changes_speed_not_tables():
    sizes = [200_000, 50_000, 9000, 4000, 100, 3 * TILE + 1, 1_000_000]
    ws = _weights(sizes, "f32", 7)
    with wrs.AliasBatch(sizes) as b:
        buf = b.pack(_to_cuda(ws))
        ms = b.tune(buf)
        assert ms > 0
        groups = b.groups()
        assert all(g in (1, 2, 4, 8) for g in groups)
        _check_tables(b, ws)
        for gs in ([1, 1, 1, 1, 1], [1, 8, 8, 8, 8], [3, 5, 7, 9, 64]):
            b.set_groups(gs)
            assert b.groups() == gs
            b.build(buf)
            assert b.status()[0] == wrs.OK
            _check_tables(b, ws)


def test_many_distribution_workload_sample():
    """A 256-table draw of the many-distribution workload (sizes log-uniform
    in [32, 2^16], k log-uniform in [1, 4096], uniform or Zipf(1.0) by seed)."""
    n, k, kinds, seeds = WL.batch_plan(256, 9, n_hi=1 << 16)
    ws = [WL.generate(kind, nt, sd, 1.0) for nt, kind, sd in zip(n, kinds, seeds)]
    with wrs.AliasBatch(n) as b:
        b.build(b.pack(_to_cuda(ws)))
        assert b.status()[0] == wrs.OK
        _check_tables(b, ws)
        b.set_samples(k)
        out = b.sample(seed=2, stream_id=0)
        torch.cuda.synchronize()
        _check_samples(b, ws, k, out, 2, 0)


def test_batch_argument_errors():
    rc, _ = wrs.batch_create([])
    assert rc == wrs.EINVAL
    rc, _ = wrs.batch_create([5, 0, 3])
    assert rc == wrs.EINVAL
    rc, _ = wrs.batch_create([1 << 32])
    assert rc == wrs.EINVAL
    with wrs.AliasBatch([10, 20]) as b:
        assert wrs.batch_sample(b.handle, 1, 0, 0, 0) == wrs.EINVAL  # never built
        assert wrs.batch_set_groups(b.handle, [0, 1, 1, 1, 1]) == wrs.EINVAL


@pytest.mark.parametrize("dtype", ["f32", "u32"])
def test_batch_of_only_one_tile_tables(dtype):
    """Every table at most one tile: the one-block whole-table builder alone
    (no tile pipeline launches); headers, light counts, buckets and samples
    equal the oracle's and the single-table path's."""
    sizes = [1, 2, 3, 7, 31, 32, 33, 255, 256, 257, 1000, 2047, 2048, 64, 1500]
    ws = _weights(sizes, dtype, 90)
    if dtype == "f32":  # degenerate shapes: all equal, one giant, subnormals, zeros
        ws[5] = np.full(32, 0.25, np.float32)
        ws[6] = np.concatenate([np.full(32, 1e-3, np.float32), np.array([1e6], np.float32)])
        ws[13] = np.array([1e-45, 3e-45, 0.0, 2.0 ** -126] * 16, np.float32)
    with wrs.AliasBatch(sizes) as b:
        b.build(b.pack(_to_cuda(ws)))
        rc, st = b.status()
        assert rc == wrs.OK and st == [wrs.OK] * len(sizes)
        _check_tables(b, ws)
        for t, w in enumerate(ws):
            qz, _ = O.build_table(w)
            with wrs.AliasTable(len(w)) as single:
                single.build(_to_cuda([w])[0])
                want = single.info()
            info = b.info(t)
            assert (info.n_light, info.light_max, info.shift) == (want.n_light, want.light_max, want.shift), t
        ks = [t * 313 + 3 for t in range(len(sizes))]
        b.set_samples(ks)
        out = b.sample(seed=5, stream_id=70)
        torch.cuda.synchronize()
        _check_samples(b, ws, ks, out, 5, 70)


def test_one_tile_table_with_a_bad_weight_fails_alone():
    sizes = [100, 2000, 5000]
    ws = _weights(sizes, "f32", 11)
    ws[0][17] = np.float32(np.nan)
    with wrs.AliasBatch(sizes) as b:
        b.build(b.pack(_to_cuda(ws)))
        rc, st = b.status()
        assert st[0] == wrs.EINVAL and st[1] == wrs.OK and st[2] == wrs.OK
        thr, alias, _ = b.download()
        for t in (1, 2):
            _, tab = O.build_table(ws[t])
            lo = b.offsets[t]
            assert np.array_equal(thr[lo:lo + sizes[t]], tab.thr)
            assert np.array_equal(alias[lo:lo + sizes[t]], tab.alias)
