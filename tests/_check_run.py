"""Runs the builders of libwrs_check.so (the library compiled with
WRS_CHECK=1) on the shapes of the parity tests and checks, besides the usual
equality with the oracle, what only the check build can show:

* every bucket of every table was stored exactly once (the build zeroes its
  buckets, each store adds one to the bucket's reserved word, so every
  reserved word must read 1): Alg. 2 and Alg. 3 give each bucket to exactly
  one step, and parity alone cannot see a bucket written twice with the same
  value;
* no index check failed (bucket indices and aliases inside the table, the
  sweep's shared-memory indices inside their window, each sweep subproblem
  ending in the heavy tile the split search gave the next one): zero failed
  checks counted and status WRS_OK.

Run as ``WRS_CHECK=1 python -m tests._check_run`` from the repository root
(the binding picks the library at import); prints one line per case and
exits non-zero on the first failure.  The GPU test that runs it is
tests/test_gpu_check.py.
"""
import sys

import numpy as np
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs
from tests import _gpu as G

TILE = 2048


def _shapes():
    rng = np.random.default_rng(202)
    cases = []
    for n in (1, 2, 3, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, 70_001):
        cases.append((f"u32_uniform_{n}", WL.u32_uniform(n, n)))
        cases.append((f"zipf1_{n}", WL.f32_zipf(n, 1.0, n + 2)))
    cases.append(("u32_uniform_1e6", WL.u32_uniform(1_000_000, 1)))
    cases.append(("f32_uniform_600013", WL.f32_uniform(600_013, 5)))
    cases.append(("zipf1.5_200000", WL.f32_zipf(200_000, 1.5, 6)))
    n = 50_000
    wide = (rng.random(n) * np.exp2(rng.integers(-30, 20, n))).astype(np.float32)
    cases.append(("f32_wide_range", wide))
    cases.append(("f32_subnormal", (rng.integers(1, 1 << 23, n) * 2.0 ** -149).astype(np.float32)))
    cases.append(("all_equal", np.full(n, 77, np.uint32)))
    g = np.ones(n, np.uint32)
    g[n // 3] = 10_000_000
    cases.append(("one_giant", g))
    z = np.zeros(n, np.uint32)
    z[::97] = 5
    cases.append(("mostly_zero", z))
    hf = np.concatenate([np.full(n // 10, 1000, np.uint32), np.ones(n - n // 10, np.uint32)])
    cases.append(("heavies_first", hf))
    cases.append(("heavies_last", hf[::-1].copy()))
    hl = np.ones(20 * TILE, np.uint32)
    hl[TILE - 1::TILE] = 3000
    cases.append(("heavy_at_each_tile_end", hl))
    cases.append(("alternating_tiles", np.repeat(np.where(np.arange(16) % 2 == 0, 1, 50).astype(np.uint32), TILE)))
    return cases


def _once(res, what):
    bad = np.nonzero(res != 1)[0]
    assert bad.size == 0, f"{what}: {bad.size} buckets not written exactly once, first {bad[:5]} counts {res[bad[:5]]}"


def _table_case(name, w, t, tab, opts=None):
    if opts is None:
        t.build(G.to_device(w))
    else:
        t.build_opts(G.to_device(w), **opts)
    st = t.status()
    assert st == wrs.OK, f"{name}: status {wrs.status_str(st)}"
    assert t.check_failures() == 0, f"{name}: {t.check_failures()} failed checks"
    thr, alias, res = t.download()
    _once(res, name)
    assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias), f"{name}: table differs from Alg. 2"


def single_tables():
    for name, w in _shapes():
        _, tab = O.build_table(w)
        with wrs.AliasTable(len(w)) as t:
            _table_case(name, w, t, tab)
        print(f"table {name}: n={len(w)} every bucket once, 0 failed checks", flush=True)


def build_options():
    w = WL.f32_zipf(3_000_007, 1.0, 41)
    _, tab = O.build_table(w)
    ntiles = (len(w) + TILE - 1) // TILE
    with wrs.AliasTable(len(w)) as t:
        for opts in ({"splits": 1}, {"splits": 3}, {"splits": 64}, {"splits": ntiles},
                     {"acc": wrs.ACC_U128}, {"splits": 7, "acc": wrs.ACC_U128}):
            _table_case(f"zipf1_3000007 {opts}", w, t, tab, opts)
            print(f"table zipf1_3000007 {opts}: every bucket once, 0 failed checks", flush=True)
        k = 2_000_000
        got = G.gpu_samples(t, k, seed=31, stream_id=(1 << 32) + 3)
        assert t.check_failures() == 0
        assert np.array_equal(got, O.sample(tab.thr, tab.alias, tab.Qp, k, 31, (1 << 32) + 3))
        print("sample zipf1_3000007: 2e6 samples equal the oracle's, 0 failed checks", flush=True)


def wide_path_at_scale():
    """n = 10^8 binary32 Zipf 1.5: Q >= 2^64, the shifted 128-bit walk."""
    n = 100_000_000
    w_dev = WL.generate_device("f32_zipf", n, 6, 1.5)
    w = w_dev.cpu().numpy()
    qz, tab = O.build_table(w)
    assert qz.Q >= 1 << 64
    with wrs.AliasTable(n) as t:
        t.build(w_dev)
        assert t.status() == wrs.OK and t.check_failures() == 0
        assert t.info().shift > 0
        thr, alias, res = t.download()
        _once(res, "zipf1.5_1e8")
        assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias)
    print(f"table zipf1.5_1e8 (shift {tab.shift}): every bucket once, 0 failed checks", flush=True)


def psa_plus():
    for name, w in _shapes()[::3] + [("zipf1.5_3000007", WL.f32_zipf(3_000_007, 1.5, 41))]:
        tab, _ = O.psa_plus(O.quantize(w), TILE, return_left=True)
        with wrs.AliasTable(len(w)) as t:
            t.build_psa_plus(G.to_device(w))
            assert t.status() == wrs.OK and t.check_failures() == 0, name
            thr, alias, res = t.download()
            _once(res, f"psa+ {name}")
            assert np.array_equal(thr, tab.thr) and np.array_equal(alias, tab.alias), name
        print(f"psa+ {name}: every bucket once, 0 failed checks", flush=True)


def batch():
    sizes = [1, 2, 3, 31, 32, 2047, 2048, 2049, 4101, 9000, 3 * TILE + 17, 70_001, 150_000, 5, 600_013]
    for dtype in ("f32", "u32"):
        ws = [WL.u32_uniform(n, 40 + t) if dtype == "u32" else
              (WL.f32_zipf(n, 1.5, 40 + t) if t % 2 else WL.f32_uniform(n, 40 + t)) for t, n in enumerate(sizes)]
        with wrs.AliasBatch(sizes) as b:
            b.build(b.pack([G.to_device(w) for w in ws]))
            rc, st = b.status()
            assert rc == wrs.OK and st == [wrs.OK] * len(sizes), st
            thr, alias, res = b.download()
            for t, w in enumerate(ws):  # the padding between tables is no bucket
                _, tab = O.build_table(w)
                lo, hi = b.offsets[t], b.offsets[t] + len(w)
                _once(res[lo:hi], f"batch {dtype} table {t}")
                assert np.array_equal(thr[lo:hi], tab.thr) and np.array_equal(alias[lo:hi], tab.alias), (dtype, t)
        print(f"batch {dtype}: {len(sizes)} tables, every bucket once, status OK", flush=True)


def two_level():
    for name, w in (("u32_3G+5", WL.u32_uniform(3 * TILE + 5, 1)), ("zipf1.5_70000", WL.f32_zipf(70_000, 1.5, 4)),
                    ("u32_5e6_three_levels", WL.u32_uniform(5_000_000, 8))):
        ref = O.build_2lvl(O.quantize(w))
        wt = torch.from_numpy(w.view(np.int32).copy() if w.dtype == np.uint32 else w.copy()).cuda()
        with wrs.AliasTable2(len(w)) as t2:
            t2.build(wt)
            assert t2.status() == wrs.OK, name
            thr, alias, res, *_ = t2.download()
            _once(res, f"2lvl {name}")
            assert np.array_equal(thr, ref.thr) and np.array_equal(alias, ref.alias), name
        print(f"2lvl {name}: {len(ref.sizes)} levels, every bucket once, status OK", flush=True)


def no_alloc():
    n = 1_000_003
    w = WL.f32_zipf(n, 1.0, 12)
    _, tab = O.build_table(w)
    buckets = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    header = torch.zeros(32, dtype=torch.int32, device="cuda")
    w_dev = G.to_device(w)
    rc = wrs.build_noalloc(w_dev.data_ptr(), n, wrs.F32, buckets.data_ptr(), header.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    assert rc == wrs.OK
    torch.cuda.synchronize()
    h = header.cpu().numpy().view(np.uint64)
    words = buckets.cpu().numpy().view(np.uint32).reshape(n, 4)
    assert int(header[0].item()) == wrs.OK
    assert int(h[8]) == 0, f"{int(h[8])} failed checks"  # reserved2[0]: byte offset 64
    _once(words[:, 3], "noalloc")
    thr = words[:, 0].astype(np.uint64) | (words[:, 1].astype(np.uint64) << np.uint64(32))
    assert np.array_equal(thr, tab.thr) and np.array_equal(words[:, 2], tab.alias)
    print("noalloc zipf1_1000003: every bucket once, 0 failed checks", flush=True)


def main():
    assert wrs.check_build() == 1, "the binding did not load libwrs_check.so (set WRS_CHECK=1)"
    for part in (single_tables, build_options, wide_path_at_scale, psa_plus, batch, two_level, no_alloc):
        part()
    print("check build: all cases passed", flush=True)


if __name__ == "__main__":
    sys.exit(main())
