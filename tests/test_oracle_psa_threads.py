"""The oracle's Alg. 3 run with its splits and packs on several host threads
(the CPU baseline of the benchmark) gives the same table as the sequential
run and as Alg. 2, for every split count tried."""
import numpy as np
import pytest

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL


@pytest.mark.parametrize("w", [WL.f32_zipf(50_000, 1.0, 3), WL.f32_uniform(40_000, 4), WL.u32_uniform(30_001, 5),
                               np.array([1, 3, 1, 3, 0, 0, 7], np.uint32)])
def test_threaded_psa_equals_sequential_and_sweep(w):
    qz, sweep = O.build_table(w)
    for p in sorted(x for x in {1, 2, 3, 7, 64, len(w) // 3 or 1, len(w)} if x <= len(w)):
        seq = O.psa(qz, p)
        t = {}
        par = O.psa_threads(qz, p, threads=4, timings=t)
        assert np.array_equal(par.bw, seq.bw) and np.array_equal(par.alias, seq.alias), p
        assert np.array_equal(par.thr, sweep.thr) and np.array_equal(par.alias, sweep.alias), p
        assert set(t) == {"begin_s", "splits_s", "packs_s", "end_s"}


def test_threaded_psa_rejects_bad_split_counts():
    qz, _ = O.build_table(np.array([1, 2, 3], np.uint32))
    with pytest.raises(O.OracleError):
        O.psa_threads(qz, 0, threads=2)
    with pytest.raises(O.OracleError):
        O.psa_threads(qz, 4, threads=2)
