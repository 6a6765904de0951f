"""n = 10^9 binary32 weights (uniform (0,1], the bench's shape and launch
configuration): properties that hold at any size, checked independently of
the CUDA kernels (PyTorch arithmetic on the downloaded table and the
weights), and sampled outputs the oracle computes one by one."""
import os

import numpy as np
import pytest
import torch

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs

pytestmark = pytest.mark.gpu

N = int(os.environ.get("WRS_FULLSIZE_N", 10 ** 9))


def test_full_size_table_and_samples():
    w = WL.generate_device("f32_uniform", N, 7)
    table = wrs.AliasTable(N)
    table.build(w)
    assert table.status() == wrs.OK
    info = table.info()
    assert info.shift == 0 and info.qp < 2 ** 62  # Q < 2^62 for these weights: int64 arithmetic below is exact
    host = np.empty(2 * N, dtype=np.uint64)
    assert wrs.table_download(table.handle, host.ctypes.data, host.nbytes) == wrs.OK
    buckets = torch.from_numpy(host.view(np.int64)).cuda()
    del host
    b = buckets.view(N, 2)
    thr = b[:, 0]
    alias = b[:, 1] & 0xFFFFFFFF
    assert int((b[:, 1] >> 32).abs().sum()) == 0
    # exact integer weights q = w * 2^-beta from the binary32 words
    bits = w.view(torch.int32).long() & 0xFFFFFFFF
    ex = (bits >> 23) & 0xFF
    m = (bits & 0x7FFFFF) | ((ex > 0).long() << 23)
    sh = torch.clamp(ex, min=1) - 150 - info.beta
    assert int(sh.max()) < 40
    q = torch.where(sh >= 0, m << sh.clamp(min=0), m >> (-sh).clamp(min=0))
    assert int(q.sum()) == info.Q
    nq = q * N
    light = bits <= info.light_max
    assert torch.equal(light, nq <= info.Q)
    assert int(light.sum()) == info.n_light
    idx = torch.arange(N, device="cuda")
    # light buckets hold their own weight; aliases are heavy items or the bucket itself
    assert torch.equal(thr[light], nq[light])
    other = alias != idx
    assert bool((~light[alias[other]]).all())
    full = thr == info.qp
    assert bool((alias[full] == idx[full]).all())
    assert bool((thr[other] < info.qp).all())
    # the pieces of every item add up to its weight n*q, exactly
    mass = thr.clone()
    mass.scatter_add_(0, alias[other], info.qp - thr[other])
    assert torch.equal(mass, nq)
    del mass, q, nq, bits, ex, m, sh, light, other, full, idx
    # 10^9 samples in the bench's configuration; 10^5 of them recomputed by the oracle
    k = 10 ** 9
    out = table.sample(k, seed=99, stream_id=3)
    pick = torch.randint(0, k, (100_000,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    got = out[pick].cpu().numpy().view(np.uint32)
    thr_h = thr.cpu().numpy().view(np.uint64)
    alias_h = alias.to(torch.int32).cpu().numpy().view(np.uint32)
    want = O.sample_at(thr_h, alias_h, info.qp, 99, 3, pick.cpu().numpy().astype(np.uint64))
    assert np.array_equal(got, want)
    table.free()
