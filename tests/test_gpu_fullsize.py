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
# host memory at the peak of a test: the downloaded 16-B buckets plus the
# oracle's copies of thresholds and aliases (28 GB at n = 10^9)
HOST_GB_NEEDED = 30.0 * N / 1e9


def _host_available_gb():
    """MemAvailable of this machine in GB, or None where it cannot be read."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024 / 1e9
    except (OSError, ValueError, IndexError):
        return None
    return None


@pytest.fixture(autouse=True)
def _enough_host_memory():
    avail = _host_available_gb()
    if avail is not None and avail < HOST_GB_NEEDED:
        pytest.skip(f"host memory: {avail:.0f} GB available, {HOST_GB_NEEDED:.0f} GB needed at n = {N}")


@pytest.mark.parametrize("builder", ["psa", "psa_plus"])
def test_full_size_table_and_samples(builder):
    """PSA (Alg. 3, the bench's headline build) and PSA+ (Sec. 4.2, per-tile
    greedy packing, then PSA on the leftovers) on the same 10^9 weights: both
    must be alias tables of the weights (light buckets hold their own weight,
    every alias is a heavy item or the bucket itself, the pieces of every item
    add up to n*q exactly), and 10^5 of 10^9 samples must equal the oracle's
    queries of the downloaded table."""
    w = WL.generate_device("f32_uniform", N, 7)
    table = wrs.AliasTable(N)
    if builder == "psa":
        table.build(w)
    else:
        table.build_psa_plus(w)
    assert table.status() == wrs.OK
    if builder == "psa_plus":
        left = table.psa_plus_leftovers()
        assert 0 < left < N // 10  # uniform weights: the tiles pack almost everything themselves
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


def test_full_size_two_level():
    """The two-level table of the same 10^9 weights: every level-0 group is an
    alias table of its members (exact mass identity on the GPU, all groups),
    300 sampled groups and the whole upper levels equal the oracle's tables,
    and 10^5 of 10^9 samples equal the oracle's walk on the same table."""
    w = WL.generate_device("f32_uniform", N, 7)
    t2 = wrs.AliasTable2(N)
    t2.build(w)
    assert t2.status() == wrs.OK
    sizes = t2.levels()
    G = wrs.TABLE2_GROUP
    assert sizes[0] == N and all(sizes[i + 1] == -(-sizes[i] // G) for i in range(len(sizes) - 1))
    nb, ng = sum(sizes), sum(-(-m // G) for m in sizes)
    host = np.empty(2 * nb, dtype=np.uint64)
    grp = np.empty(2 * ng, dtype=np.uint64)
    assert wrs.table2_download(t2.handle, host.ctypes.data, host.nbytes, grp.ctypes.data, grp.nbytes) == wrs.OK
    thr_all = host.reshape(nb, 2)[:, 0]
    word1 = host.reshape(nb, 2)[:, 1]
    alias_all = (word1 & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert not (word1 >> np.uint64(32)).any()
    qp_all = grp.reshape(ng, 2)[:, 0]
    sh_all = (grp.reshape(ng, 2)[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    g0 = -(-N // G)
    # exact q: the uniform recipe's weights are k * 2^-24, k in [1, 2^24]
    q = (w.double() * 2.0 ** 24).long()
    assert bool((q >= 1).all()) and bool((q <= 2 ** 24).all())
    pad = g0 * G - N
    qg = torch.cat([q, torch.zeros(pad, dtype=torch.long, device="cuda")]).view(g0, G)
    totals = qg.sum(dim=1)  # exact: < 2^35
    assert np.array_equal(qp_all[:g0], totals.cpu().numpy().astype(np.uint64)) and not sh_all[:g0].any()
    # every level-0 group: light buckets hold their weight, pieces add up to n_g * q
    thr = torch.from_numpy(thr_all[:N].view(np.int64)).cuda()
    alias = torch.from_numpy(alias_all[:N].astype(np.int64)).cuda()
    idx = torch.arange(N, device="cuda")
    gid = idx // G
    ngm = torch.full((g0,), G, dtype=torch.long, device="cuda")
    ngm[-1] = N - (g0 - 1) * G
    nq = q * ngm[gid]
    qpb = totals[gid]
    assert bool((gid[alias] == gid).all()), "an alias leaves its group"
    light = nq <= qpb
    assert torch.equal(thr[light], nq[light])
    other = alias != idx
    assert bool((~light[alias[other]]).all())
    mass = thr.clone()
    mass.scatter_add_(0, alias[other], qpb[other] - thr[other])
    assert torch.equal(mass, nq)
    del thr, alias, idx, gid, nq, qpb, light, other, mass
    # 300 sampled level-0 groups (and the ragged last one) against the oracle's Alg. 2
    gen = np.random.default_rng(17)
    qh = q.cpu().numpy()
    for g in list(gen.choice(g0 - 1, 300, replace=False)) + [g0 - 1]:
        b0, m = g * G, min(G, N - g * G)
        qq = np.zeros((m, 2), np.uint64)
        qq[:, 0] = qh[b0:b0 + m].astype(np.uint64)
        Qg = int(qh[b0:b0 + m].sum())
        tab = O.sweep(O.Quantized(qq, np.array([Qg, 0], np.uint64), 0))
        assert np.array_equal(thr_all[b0:b0 + m], tab.thr), g
        assert np.array_equal(alias_all[b0:b0 + m].astype(np.int64) - b0, tab.alias.astype(np.int64)), g
    # the upper levels: the oracle's two-level table over the group totals
    tq = np.zeros((g0, 2), np.uint64)
    tq[:, 0] = totals.cpu().numpy().astype(np.uint64)
    upper = O.build_2lvl(O.Quantized(tq, np.array([int(tq[:, 0].sum()), 0], np.uint64), 0))
    assert upper.sizes == sizes[1:]
    assert np.array_equal(thr_all[N:], upper.thr) and np.array_equal(alias_all[N:], upper.alias)
    assert np.array_equal(qp_all[g0:], upper.qp) and np.array_equal(sh_all[g0:], upper.shift)
    del q, qg, qh
    # 10^9 samples; 10^5 of them walked by the oracle on the downloaded table
    k = 10 ** 9
    out = t2.sample(k, seed=99, stream_id=3)
    pick = torch.randint(0, k, (100_000,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(6))
    got = out[pick].cpu().numpy().view(np.uint32)
    walk = O.TwoLevel(N, G, sizes, np.ascontiguousarray(thr_all), np.ascontiguousarray(alias_all),
                      np.ascontiguousarray(qp_all), sh_all, None)
    want = O.sample_2lvl_at(walk, 99, 3, pick.cpu().numpy().astype(np.uint64))
    assert np.array_equal(got, want)
    t2.free()


def test_full_size_zipf15_shifted_coin():
    """n = 10^9 binary32 Zipf 1.5 weights (the bench's third input): Q is near
    2^69, so thresholds are shifted (thr = bw >> s, s > 0) and the build runs
    on its 128-bit path.  Checked: the header against Python's exact sum;
    10^6 sampled light buckets hold (n q) >> s exactly; every bucket's alias
    is a heavy item or itself, full buckets point to themselves; and 10^5 of
    10^9 samples equal the oracle's queries of the downloaded table."""
    w = WL.generate_device("f32_zipf", N, 6, 1.5)
    table = wrs.AliasTable(N)
    table.build(w)
    assert table.status() == wrs.OK
    info = table.info()
    assert info.shift > 0
    host = np.empty(2 * N, dtype=np.uint64)
    assert wrs.table_download(table.handle, host.ctypes.data, host.nbytes) == wrs.OK
    thr_h = np.ascontiguousarray(host.reshape(N, 2)[:, 0])
    word1 = host.reshape(N, 2)[:, 1]
    alias_h = (word1 & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert not (word1 >> np.uint64(32)).any()
    del host, word1
    bits = w.view(torch.int32).cpu().numpy().view(np.uint32)
    light = bits <= np.uint32(info.light_max)
    assert int(light.sum()) == info.n_light
    # light buckets: exact n*q >> s on a sample, with Python integers
    rng = np.random.default_rng(3)
    lights = np.nonzero(light)[0]
    pick = rng.choice(lights, 1_000_000, replace=False)
    for i in pick[:20_000].tolist():  # Python big ints: the slow, obviously exact form
        x = int(bits[i])
        ex, m = (x >> 23) & 0xFF, x & 0x7FFFFF
        if ex:
            m |= 1 << 23
        e = (ex if ex else 1) - 150 - info.beta
        q = m << e if e >= 0 else m >> -e
        assert int(thr_h[i]) == (N * q) >> info.shift, i
    # the whole sample: q as exact integers (a light's q is below Q / n), then
    # (N * q) >> s in Python integers
    xs = bits[pick].astype(np.int64)
    ex = (xs >> 23) & 0xFF
    m = (xs & 0x7FFFFF) | (np.where(ex > 0, 1, 0) << 23)
    e = np.where(ex > 0, ex, 1) - 150 - info.beta
    assert e.max() <= 30
    q = np.where(e >= 0, m << np.maximum(e, 0), m >> np.maximum(-e, 0)).astype(object)
    got = thr_h[pick].astype(object)
    want = (q * N) >> info.shift
    assert (got == want).all()
    # aliases: a heavy item or the bucket itself; full buckets point to themselves
    idx = np.arange(N, dtype=np.uint32)
    other = alias_h != idx
    assert (~light[alias_h[other]]).all()
    full = thr_h == np.uint64(info.qp)
    assert (alias_h[full] == idx[full]).all()
    assert (thr_h[other] < np.uint64(info.qp)).all()
    del idx, other, full, light, bits, xs, m, e, q
    # 10^9 samples; 10^5 of them recomputed by the oracle
    k = 10 ** 9
    out = table.sample(k, seed=77, stream_id=1)
    sel = torch.randint(0, k, (100_000,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(9))
    got_s = out[sel].cpu().numpy().view(np.uint32)
    want_s = O.sample_at(thr_h, alias_h, info.qp, 77, 1, sel.cpu().numpy().astype(np.uint64))
    assert np.array_equal(got_s, want_s)
    table.free()
