"""wrs_build_noalloc: the build for callers that cannot allocate device
memory (real-time processes with a device memory budget fixed at start-up,
frameworks that own all device memory through their own pool).  It must produce, through the C ABI, exactly the buckets
and header values of the ordinary build, call after call, although every call
reuses the library's one static scratch array.  This file is collected last
so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _noalloc(w_dev, n, dtype, stream):
    buckets = torch.zeros(2 * n, dtype=torch.int64, device="cuda")  # n x 16 bytes, 16-B aligned
    header = torch.zeros(wrs.DEVICE_HEADER_BYTES // 8, dtype=torch.int64, device="cuda")
    rc = wrs.build_noalloc(w_dev.data_ptr(), n, dtype, buckets.data_ptr(), header.data_ptr(), stream)
    assert rc == wrs.OK, wrs.status_str(rc)
    torch.cuda.synchronize()
    b = buckets.cpu().numpy().view(np.uint64).reshape(n, 2)
    h = header.cpu().numpy().view(np.uint64)
    thr = b[:, 0].copy()
    alias = (b[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    reserved = (b[:, 1] >> np.uint64(32)).astype(np.uint32)
    status = int(h[0] & np.uint64(0xFFFFFFFF))
    return thr, alias, reserved, status, h


def test_noalloc_matches_the_ordinary_build_two_calls_in_a_row():
    stream = torch.cuda.current_stream().cuda_stream
    cases = [WL.f32_zipf(300_001, 1.0, 21), WL.u32_uniform(1_048_579, 22)]
    results = []
    for w in cases:  # two calls in a row, different inputs and dtypes
        n = len(w)
        dtype = wrs.F32 if w.dtype == np.float32 else wrs.U32
        w_dev = G.to_device(w)
        thr, alias, reserved, status, h = _noalloc(w_dev, n, dtype, stream)
        with wrs.AliasTable(n) as t:
            t.build(w_dev)
            assert t.status() == wrs.OK
            want_thr, want_alias, _ = t.download()
            info = t.info()
        assert status == wrs.OK
        assert np.array_equal(thr, want_thr) and np.array_equal(alias, want_alias)
        assert not reserved.any()
        q = int(h[2]) | (int(h[3]) << 64)
        assert q == info.Q and int(h[4]) == info.qp
        results.append((thr, alias))
    # the first input again: the shared scratch keeps no state between calls
    w = cases[0]
    thr, alias, _, status, _ = _noalloc(G.to_device(w), len(w), wrs.F32, stream)
    assert status == wrs.OK
    assert np.array_equal(thr, results[0][0]) and np.array_equal(alias, results[0][1])


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    n = wrs.NOALLOC_MAX_N + 1
    rc = wrs.build_noalloc(ctypes.c_void_p(16).value, n, wrs.F32, 16, 16, 0)
    assert rc == wrs.EINVAL
