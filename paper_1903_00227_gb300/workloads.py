"""Seeded synthetic weight generators (shared input recipe; no method arithmetic).

The paper's inputs (Sec. 10, paragraph "Input Data") are uniform random weights
in (0, 1] and random permutations of {1^-s, 2^-s, ..., n^-s}.  This module
fixes one reproducible recipe for them and for uint32 weights:

* every random word is SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) of a
  counter: ``x_i = splitmix64(base + i)`` with ``base = splitmix64(seed ^
  (purpose << 48))``;
* ``u32_uniform``: w_i = 1 + (x_i & 0xFFFFFF), i.e. uniform on [1, 2^24];
* ``f32_uniform``: w_i = (1 + (x_i >> 40)) * 2^-24, uniform on the 2^-24 grid
  of (0, 1] (exact in binary32);
* ``f32_zipf``: w_i = fl32((pi(i) + 1)^-s), pi a seeded bijection of [0, n)
  (a four-round balanced Feistel network on 2h >= log2 n bits, restricted to
  [0, n) by cycle walking, Black and Rogaway, CT-RSA 2002).

Both the oracle and the CUDA library receive the same array: it is generated
once, on the host here or on the device by ``libwrs_workloads.so`` (same
recipe; ``f32_zipf``'s power may round differently there in rare last bits, so
a device-made array is copied to the host when the oracle needs it).  This
module holds none of the alias-table arithmetic.
"""
from __future__ import annotations

import numpy as np

_M = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _base(seed: int, purpose: int) -> np.uint64:
    s = np.uint64((seed ^ (purpose << 48)) & 0xFFFFFFFFFFFFFFFF)
    return splitmix64(np.array([s], dtype=np.uint64))[0]


def words(n: int, seed: int, purpose: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        return splitmix64(_base(seed, purpose) + np.arange(n, dtype=np.uint64))


PURPOSE_VALUE = 1
PURPOSE_PERM = 2


def u32_uniform(n: int, seed: int) -> np.ndarray:
    x = words(n, seed, PURPOSE_VALUE)
    return (np.uint64(1) + (x & np.uint64(0xFFFFFF))).astype(np.uint32)


def f32_uniform(n: int, seed: int) -> np.ndarray:
    x = words(n, seed, PURPOSE_VALUE)
    m = (np.uint64(1) + (x >> np.uint64(40))).astype(np.float64)
    return (m * 2.0 ** -24).astype(np.float32)


def feistel_half_bits(n: int) -> int:
    bits = max(1, int(n - 1).bit_length())
    return max(1, (bits + 1) // 2)


def _feistel(x: np.ndarray, h: int, keys: np.ndarray) -> np.ndarray:
    mask = np.uint64((1 << h) - 1)
    L = x >> np.uint64(h)
    R = x & mask
    for k in keys:
        L, R = R, L ^ (splitmix64(k ^ R) & mask)
    return (L << np.uint64(h)) | R


def permutation(n: int, seed: int) -> np.ndarray:
    """pi(0..n-1): a seeded bijection of [0, n) (Feistel + cycle walking)."""
    h = feistel_half_bits(n)
    keys = words(4, seed, PURPOSE_PERM)
    y = _feistel(np.arange(n, dtype=np.uint64), h, keys)
    out_of_range = y >= np.uint64(n)
    while out_of_range.any():
        y[out_of_range] = _feistel(y[out_of_range], h, keys)
        out_of_range = y >= np.uint64(n)
    return y


def f32_zipf(n: int, s: float, seed: int) -> np.ndarray:
    r = permutation(n, seed).astype(np.float64) + 1.0
    return np.power(r, -float(s)).astype(np.float32)


def generate(kind: str, n: int, seed: int, s: float = 1.0) -> np.ndarray:
    if kind == "u32_uniform":
        return u32_uniform(n, seed)
    if kind == "f32_uniform":
        return f32_uniform(n, seed)
    if kind == "f32_zipf":
        return f32_zipf(n, s, seed)
    raise ValueError(kind)


# ------------------------------------------------------- many distributions
PURPOSE_BATCH = 3


def log_uniform_ints(count: int, lo: int, hi: int, seed: int, purpose: int) -> np.ndarray:
    """count integers log-uniform on [lo, hi]: floor(lo * (hi + 1 / lo)^u), u
    the top 53 bits of a SplitMix64 word, clipped to [lo, hi]."""
    u = (words(count, seed, purpose) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    v = np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo))))
    return np.clip(v, lo, hi).astype(np.int64)


def batch_plan(ntables: int, seed: int, n_lo: int = 32, n_hi: int = 1 << 20, k_lo: int = 1, k_hi: int = 4096):
    """Many independent distributions: per table its size n (log-uniform in
    [n_lo, n_hi]), its sample count k (log-uniform in [k_lo, k_hi]), its kind
    (binary32 uniform or Zipf s = 1.0, one random bit) and its weight seed."""
    n = log_uniform_ints(ntables, n_lo, n_hi, seed, PURPOSE_BATCH)
    k = log_uniform_ints(ntables, k_lo, k_hi, seed ^ 0x5A5A5A5A, PURPOSE_BATCH)
    bit = words(ntables, seed ^ 0xA5A5A5A5, PURPOSE_BATCH) & np.uint64(1)
    kinds = ["f32_zipf" if b else "f32_uniform" for b in bit]
    seeds = [int(seed) * 1_000_003 + t for t in range(ntables)]
    return [int(x) for x in n], [int(x) for x in k], kinds, seeds


# --------------------------------------------------------------- device side
KINDS = {"u32_uniform": 0, "f32_uniform": 1, "f32_zipf": 2}
_wl = None


def _wl_lib():
    global _wl
    if _wl is None:
        import ctypes
        import os

        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libwrs_workloads.so")
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        lib.wl_generate.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_double, ctypes.c_void_p]
        lib.wl_generate.restype = ctypes.c_int
        lib.wl_random_gather.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_void_p]
        lib.wl_random_gather.restype = ctypes.c_int
        _wl = lib
    return _wl


def generate_device(kind: str, n: int, seed: int, s: float = 1.0, out=None, stream=None):
    """Same recipe as ``generate`` but computed on the GPU into a torch tensor
    (float32 for the f32 kinds, int32 words for u32_uniform)."""
    import torch

    dt = torch.int32 if kind == "u32_uniform" else torch.float32
    if out is None:
        out = torch.empty(n, dtype=dt, device="cuda")
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = _wl_lib().wl_generate(KINDS[kind], out.data_ptr(), n, seed, float(s), st)
    if rc:
        raise RuntimeError(f"wl_generate failed ({rc})")
    return out


def random_gather(d_table: int, n: int, k: int, seed: int, d_out: int, stream: int) -> None:
    """k random 16-byte gathers from a device table of n entries (measurement
    of the random-access ceiling that bounds alias sampling)."""
    rc = _wl_lib().wl_random_gather(d_table, n, k, seed, d_out, stream)
    if rc:
        raise RuntimeError(f"wl_random_gather failed ({rc})")
