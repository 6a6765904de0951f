"""The build's wide path at scale: n = 10^8 binary32 Zipf 1.5 weights
(randomly permuted, seed 6).  Their exact total Q is above 2^64, so the
thresholds are shifted (shift > 0) and the sweep runs its 128-bit walk; the
table must still equal the oracle's Alg. 2 bucket for bucket (thresholds and
aliases), with the same header, and 10^7 samples must equal the oracle's."""
import numpy as np
import pytest

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL
from paper_1903_00227_gb300 import wrs
from tests import _gpu as G

pytestmark = pytest.mark.gpu

N = 100_000_000


def test_n1e8_zipf15_shifted_path_is_bucket_exact():
    w_dev = WL.generate_device("f32_zipf", N, 6, 1.5)
    w = w_dev.cpu().numpy()
    qz, tab = O.build_table(w)
    assert qz.Q >= 1 << 64  # the wide path is the one under test
    with wrs.AliasTable(N) as t:
        t.build(w_dev)
        assert t.status() == wrs.OK
        info = t.info()
        assert info.Q == qz.Q and info.beta == qz.beta
        assert info.shift == tab.shift > 0 and info.qp == tab.Qp
        T = qz.Q // N  # light iff n * q <= Q iff q <= floor(Q / n) (Sec. 2.2, ties light)
        t_hi, t_lo = np.uint64(T >> 64), np.uint64(T & ((1 << 64) - 1))
        q_lo, q_hi = qz.q[:, 0], qz.q[:, 1]
        n_light = int(np.count_nonzero((q_hi < t_hi) | ((q_hi == t_hi) & (q_lo <= t_lo))))
        assert info.n_light == n_light
        thr, alias, reserved = t.download()
        assert np.array_equal(thr, tab.thr), int(np.count_nonzero(thr != tab.thr))
        assert np.array_equal(alias, tab.alias), int(np.count_nonzero(alias != tab.alias))
        assert not reserved.any()
        k = 10_000_000
        got = G.gpu_samples(t, k, seed=606, stream_id=(1 << 32) + 9)
    want = O.sample(tab.thr, tab.alias, tab.Qp, k, 606, (1 << 32) + 9)
    assert np.array_equal(got, want)
