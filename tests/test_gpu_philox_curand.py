"""The oracle's Philox4x32-10 against an independent implementation: cuRAND's
device function curand_Philox4x32_10, called (not copied) on a grid of
counters and keys."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import wrs_oracle as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_matches_curand(tmp_path):
    so = str(tmp_path / "curand_philox.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, os.path.join(HERE, "curand_philox.cu")])
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(7)
    m = 4096
    ctr = rng.integers(0, 2 ** 32, size=(m, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(m, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 1, 0]]
    out = np.zeros((m, 4), dtype=np.uint32)
    assert lib.curand_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, m) == 0
    for i in range(m):
        assert O.philox(ctr[i].tolist(), key[i].tolist()) == tuple(int(v) for v in out[i]), i
