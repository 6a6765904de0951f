"""ctypes front end of the C oracle in ``wrs_oracle.c`` (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing here is shared
with the CUDA library.  Every function follows a passage of L.
Huebschle-Schneider and P. Sanders, "Parallel Weighted Random Sampling":

* ``quantize``   -- W = sum w_i (first line of Alg. 1/2/3) in exact integer units
* ``sweep``      -- Alg. 2, the sweeping construction (Sec. 4.1)
* ``psa``        -- Alg. 3, split + pack (Sec. 4.2)
* ``vose``       -- Alg. 1, Vose-style construction (Sec. 2.2), exact integers
* ``vose_f64``   -- Alg. 1 in binary64, the paper's sequential baseline
* ``encode``     -- the 64-bit coin thresholds of the table
* ``philox``     -- Philox4x32-10 (Salmon et al., SC 2011)
* ``sample``     -- k alias queries (Sec. 2.2, Sec. 5 Cor. "kWR")

Parity is pinned for every function by the tests in ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force and hand-worked examples).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wrs_oracle.c")
LIB = os.path.join(HERE, "libwrs_oracle.so")

OK, EINVAL, EOVERFLOW, EINTERNAL = 0, 1, 2, 3
U32, F32 = 0, 1

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"oracle {where} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/libwrs_oracle.so``."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            P = ctypes.c_void_p
            U64, I32, INT = ctypes.c_uint64, ctypes.c_int32, ctypes.c_int
            L.wo_quantize.argtypes = [INT, P, U64, P, P, P]
            L.wo_quantize.restype = INT
            for f in (L.wo_sweep, L.wo_vose):
                f.argtypes = [U64, P, P, P, P]
                f.restype = INT
            L.wo_psa.argtypes = [U64, P, P, U64, P, P, P]
            L.wo_psa.restype = INT
            L.wo_vose_f64.argtypes = [U64, P, P, P]
            L.wo_vose_f64.restype = INT
            L.wo_encode.argtypes = [U64, P, P, P, P, P]
            L.wo_encode.restype = None
            L.wo_philox4x32_10.argtypes = [P, P, P]
            L.wo_philox4x32_10.restype = None
            L.wo_sample.argtypes = [U64, P, P, U64, U64, U64, U64, P]
            L.wo_sample.restype = None
            L.wo_sample_at.argtypes = [U64, P, P, U64, U64, U64, P, U64, P]
            L.wo_sample_at.restype = None
            L.wo_2lvl_levels.argtypes = [U64, U64, P]
            L.wo_2lvl_levels.restype = INT
            L.wo_2lvl_build.argtypes = [U64, P, U64, P, P, P, P, P]
            L.wo_2lvl_build.restype = INT
            L.wo_2lvl_sample.argtypes = [U64, U64, P, P, P, U64, U64, U64, P]
            L.wo_2lvl_sample.restype = None
            L.wo_2lvl_sample_at.argtypes = [U64, U64, P, P, P, U64, U64, P, U64, P]
            L.wo_2lvl_sample_at.restype = None
            L.wo_os_nd.argtypes = [U64, U64, P, P, P, P, P, U64, U64, U64, P, P, U64]
            L.wo_os_nd.restype = U64
            L.wo_binomial.argtypes = [U64, U64, U64, U64, U64]
            L.wo_binomial.restype = U64
            L.wo_det_log.argtypes = [ctypes.c_double]
            L.wo_det_log.restype = ctypes.c_double
            L.wo_det_exp.argtypes = [ctypes.c_double]
            L.wo_det_exp.restype = ctypes.c_double
            L.wo_det_log1m.argtypes = [ctypes.c_double]
            L.wo_det_log1m.restype = ctypes.c_double
            L.wo_det_lfact.argtypes = [U64]
            L.wo_det_lfact.restype = ctypes.c_double
            L.wo_det_u128_to_double.argtypes = [U64, U64]
            L.wo_det_u128_to_double.restype = ctypes.c_double
            L.wo_det_ldexp.argtypes = [ctypes.c_double, INT]
            L.wo_det_ldexp.restype = ctypes.c_double
            L.wo_psa_plus.argtypes = [U64, P, P, U64, P, P, P]
            L.wo_psa_plus.restype = INT
            L.wo_psa_begin.argtypes = [U64, P, P, U64, P, P]
            L.wo_psa_begin.restype = P
            for f in (L.wo_psa_split, L.wo_psa_pack):
                f.argtypes = [P, U64]
                f.restype = INT
            L.wo_psa_end.argtypes = [P, P]
            L.wo_psa_end.restype = None
            L.wo_psa_free.argtypes = [P]
            L.wo_psa_free.restype = None
            _lib = L
    return _lib


class use_library:
    """Run the oracle functions of this module against another build of
    wrs_oracle.c (used by the tests that plant mistakes in the oracle)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()  # configure the default library first
        self.saved = _lib
        L = ctypes.CDLL(self.path)
        for name in ("wo_quantize", "wo_sweep", "wo_vose", "wo_psa", "wo_vose_f64", "wo_encode",
                     "wo_philox4x32_10", "wo_sample", "wo_sample_at", "wo_2lvl_levels", "wo_2lvl_build",
                     "wo_2lvl_sample", "wo_2lvl_sample_at", "wo_os_nd", "wo_binomial", "wo_det_log",
                     "wo_det_exp", "wo_det_log1m", "wo_det_lfact", "wo_det_u128_to_double", "wo_det_ldexp",
                     "wo_psa_plus"):
            f, g = getattr(L, name), getattr(self.saved, name)
            f.argtypes, f.restype = g.argtypes, g.restype
        with _lock:
            _lib = L
        return L

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def u128_to_int(words: np.ndarray) -> int:
    return int(words[0]) | (int(words[1]) << 64)


def to_words(a: np.ndarray) -> np.ndarray:
    """Weights as raw 32-bit words (binary32 patterns are passed by bits)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.float32:
        return a.view(np.uint32)
    if a.dtype == np.uint32:
        return a
    raise TypeError(f"weights must be uint32 or float32, got {a.dtype}")


def dtype_code(a: np.ndarray) -> int:
    return F32 if a.dtype == np.float32 else U32


class Quantized:
    """Exact integer weights: q[i] (two uint64 words each), Q, beta."""

    def __init__(self, q: np.ndarray, Qw: np.ndarray, beta: int):
        self.q, self.Qw, self.beta = q, Qw, beta

    @property
    def n(self) -> int:
        return self.q.shape[0]

    @property
    def Q(self) -> int:
        return u128_to_int(self.Qw)

    def q_int(self, i: int) -> int:
        return u128_to_int(self.q[i])


def quantize(w: np.ndarray) -> Quantized:
    words = to_words(w)
    n = words.shape[0]
    q = np.zeros((max(n, 1), 2), dtype=np.uint64)
    Qw = np.zeros(2, dtype=np.uint64)
    beta = ctypes.c_int32(0)
    rc = lib().wo_quantize(dtype_code(w), _ptr(words), n, _ptr(q), _ptr(Qw), ctypes.addressof(beta))
    if rc:
        raise OracleError(rc, "quantize")
    return Quantized(q[:n], Qw, beta.value)


class Table:
    """An alias table: exact bucket masses bw (two words each), aliases, and
    the encoded coin thresholds thr with Qp and shift."""

    def __init__(self, bw: np.ndarray, alias: np.ndarray, Qw: np.ndarray):
        self.bw, self.alias, self.Qw = bw, alias, Qw
        n = alias.shape[0]
        self.thr = np.zeros(n, dtype=np.uint64)
        qp = ctypes.c_uint64(0)
        sh = ctypes.c_uint32(0)
        lib().wo_encode(n, _ptr(bw), _ptr(Qw), _ptr(self.thr), ctypes.addressof(qp), ctypes.addressof(sh))
        self.Qp, self.shift = qp.value, sh.value

    @property
    def n(self) -> int:
        return self.alias.shape[0]

    def bw_int(self, b: int) -> int:
        return u128_to_int(self.bw[b])


def _construct(fn, qz: Quantized, *extra) -> Table:
    n = qz.n
    bw = np.zeros((n, 2), dtype=np.uint64)
    al = np.zeros(n, dtype=np.uint32)
    rc = fn(n, _ptr(qz.q), _ptr(qz.Qw), *extra, _ptr(bw), _ptr(al))
    if rc:
        raise OracleError(rc, fn.__name__)
    return Table(bw, al, qz.Qw)


def psa_plus(qz: Quantized, T: int = 2048, return_left: bool = False):
    """PSA+ (Sec. 4.2 "Performance Optimization in Practice") with tiles of T
    items; optionally also the number of items left to the second phase."""
    n = qz.n
    bw = np.zeros((n, 2), dtype=np.uint64)
    al = np.zeros(n, dtype=np.uint32)
    left = ctypes.c_uint64(0)
    rc = lib().wo_psa_plus(n, _ptr(qz.q), _ptr(qz.Qw), T, _ptr(bw), _ptr(al), ctypes.addressof(left))
    if rc:
        raise OracleError(rc, "psa_plus")
    t = Table(bw, al, qz.Qw)
    return (t, left.value) if return_left else t


def sweep(qz: Quantized) -> Table:
    return _construct(lib().wo_sweep, qz)


def vose(qz: Quantized) -> Table:
    return _construct(lib().wo_vose, qz)


def psa(qz: Quantized, p: int, return_splits: bool = False):
    n = qz.n
    bw = np.zeros((n, 2), dtype=np.uint64)
    al = np.zeros(n, dtype=np.uint32)
    splits = np.zeros((p + 1, 4), dtype=np.uint64)
    rc = lib().wo_psa(n, _ptr(qz.q), _ptr(qz.Qw), p, _ptr(bw), _ptr(al), _ptr(splits))
    if rc:
        raise OracleError(rc, "psa")
    t = Table(bw, al, qz.Qw)
    return (t, splits) if return_splits else t


def psa_threads(qz: Quantized, p: int, threads: int, timings: dict | None = None) -> Table:
    """Alg. 3 with its p - 1 splits and p packs run on `threads` host
    threads (the oracle's own split and pack steps, unchanged; each call
    releases the interpreter lock).  The table equals psa(qz, p)'s.  When
    `timings` is a dict it receives the seconds of each phase."""
    import time
    from concurrent.futures import ThreadPoolExecutor

    n = qz.n
    L = lib()
    bw = np.zeros((n, 2), dtype=np.uint64)
    al = np.zeros(n, dtype=np.uint32)
    t0 = time.perf_counter()
    ctx = L.wo_psa_begin(n, _ptr(qz.q), _ptr(qz.Qw), p, _ptr(bw), _ptr(al))
    if not ctx:
        raise OracleError(1, "psa_begin")
    t1 = time.perf_counter()
    try:
        def run(fn, ks):
            rcs = [fn(ctx, k) for k in ks]
            bad = [rc for rc in rcs if rc]
            return bad[0] if bad else 0

        with ThreadPoolExecutor(max_workers=threads) as ex:
            parts = lambda lo, hi: [range(lo + i, hi, threads) for i in range(threads)]
            rc = max(ex.map(lambda ks: run(L.wo_psa_split, ks), parts(1, p)), default=0)
            t2 = time.perf_counter()
            if rc == 0:
                rc = max(ex.map(lambda ks: run(L.wo_psa_pack, ks), parts(1, p + 1)), default=0)
        t3 = time.perf_counter()
    except BaseException:
        L.wo_psa_free(ctx)
        raise
    if rc:
        L.wo_psa_free(ctx)
        raise OracleError(rc, "psa_threads")
    L.wo_psa_end(ctx, None)
    t4 = time.perf_counter()
    if timings is not None:
        timings.update({"begin_s": t1 - t0, "splits_s": t2 - t1, "packs_s": t3 - t2, "end_s": t4 - t3})
    return Table(bw, al, qz.Qw)


def vose_f64(w: np.ndarray):
    wd = np.ascontiguousarray(w, dtype=np.float64)
    n = wd.shape[0]
    prob = np.zeros(n, dtype=np.float64)
    al = np.zeros(n, dtype=np.uint32)
    rc = lib().wo_vose_f64(n, _ptr(wd), _ptr(prob), _ptr(al))
    if rc:
        raise OracleError(rc, "vose_f64")
    return prob, al


def philox(ctr, key) -> tuple:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().wo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return tuple(int(x) for x in out)


def sample(thr: np.ndarray, alias: np.ndarray, Qp: int, k: int, seed: int, stream: int = 0) -> np.ndarray:
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    alias = np.ascontiguousarray(alias, dtype=np.uint32)
    out = np.zeros(max(k, 1), dtype=np.uint32)
    lib().wo_sample(thr.shape[0], _ptr(thr), _ptr(alias), Qp, k, seed, stream, _ptr(out))
    return out[:k]


def build_table(w: np.ndarray) -> tuple:
    """quantize + sweep: the table the CUDA build must reproduce bit for bit."""
    qz = quantize(w)
    return qz, sweep(qz)


def sample_at(thr: np.ndarray, alias: np.ndarray, Qp: int, seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """The queries of ``sample`` for the sample indices ``idx`` only."""
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    alias = np.ascontiguousarray(alias, dtype=np.uint32)
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.zeros(max(idx.shape[0], 1), dtype=np.uint32)
    lib().wo_sample_at(thr.shape[0], _ptr(thr), _ptr(alias), Qp, seed, stream, _ptr(idx), idx.shape[0], _ptr(out))
    return out[: idx.shape[0]]


# ------------------------------------------------- two-level ("2lvl-sweep") tables
GROUP = 2048  # members per group at every level


class TwoLevel:
    """Multi-level table (Sec. 6, replicated top level, Alg. 2 per group):
    per level, thresholds and aliases (alias = member index within the level);
    per group (level 0's groups first), qp, shift and the exact group total."""

    def __init__(self, n: int, G: int, sizes, thr, alias, qp, shift, tot):
        self.n, self.G, self.sizes = n, G, list(sizes)
        self.thr, self.alias, self.qp, self.shift, self.tot = thr, alias, qp, shift, tot

    @property
    def levels(self) -> int:
        return len(self.sizes)

    def level_slice(self, level: int) -> slice:
        o = sum(self.sizes[:level])
        return slice(o, o + self.sizes[level])

    def group_slice(self, level: int) -> slice:
        o = sum((m + self.G - 1) // self.G for m in self.sizes[:level])
        return slice(o, o + (self.sizes[level] + self.G - 1) // self.G)


def levels_2lvl(n: int, G: int = GROUP):
    sizes = np.zeros(16, dtype=np.uint64)
    L = lib().wo_2lvl_levels(n, G, _ptr(sizes))
    return [int(x) for x in sizes[:L]]


def build_2lvl(qz: Quantized, G: int = GROUP) -> TwoLevel:
    n = qz.n
    sizes = levels_2lvl(n, G)
    total = sum(sizes)
    groups = sum((m + G - 1) // G for m in sizes)
    thr = np.zeros(total, dtype=np.uint64)
    al = np.zeros(total, dtype=np.uint32)
    qp = np.zeros(groups, dtype=np.uint64)
    sh = np.zeros(groups, dtype=np.uint32)
    tot = np.zeros((groups, 2), dtype=np.uint64)
    rc = lib().wo_2lvl_build(n, _ptr(qz.q), G, _ptr(thr), _ptr(al), _ptr(qp), _ptr(sh), _ptr(tot))
    if rc:
        raise OracleError(rc, "2lvl_build")
    return TwoLevel(n, G, sizes, thr, al, qp, sh, tot)


def sample_2lvl(t: TwoLevel, k: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(max(k, 1), dtype=np.uint32)
    lib().wo_2lvl_sample(t.n, t.G, _ptr(t.thr), _ptr(t.alias), _ptr(t.qp), k, seed, stream, _ptr(out))
    return out[:k]


def sample_2lvl_at(t: TwoLevel, seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.zeros(max(idx.shape[0], 1), dtype=np.uint32)
    lib().wo_2lvl_sample_at(t.n, t.G, _ptr(t.thr), _ptr(t.alias), _ptr(t.qp), seed, stream, _ptr(idx),
                            idx.shape[0], _ptr(out))
    return out[: idx.shape[0]]


# ------------------------------------------------- output-sensitive sampling (OS-ND)
def os_nd(qz: Quantized, t: TwoLevel, k: int, seed: int, stream: int = 0, cap: int | None = None):
    """(items, counts) of OS-ND sampling k items with replacement over the
    two-level table t of the exact weights qz (pairs in the order drawn)."""
    if cap is None:
        cap = min(k, qz.n + 128 * (qz.n // t.G + 1)) + 1
    items = np.zeros(max(cap, 1), dtype=np.uint32)
    counts = np.zeros(max(cap, 1), dtype=np.uint64)
    m = lib().wo_os_nd(qz.n, t.G, _ptr(qz.q), _ptr(t.thr), _ptr(t.alias), _ptr(t.qp), _ptr(t.tot), k, seed,
                       stream, _ptr(items), _ptr(counts), cap)
    if m == 2 ** 64 - 1:
        raise OracleError(-1, "os_nd (output capacity)")
    return items[:m], counts[:m]


def binomial(n: int, num: int, den: int, seed: int, node: int) -> int:
    """One Binomial(n, num/den) deviate of the OS-ND generator (node = draw stream)."""
    return int(lib().wo_binomial(n, num, den, seed, node))


def det_log(x: float) -> float:
    return float(lib().wo_det_log(x))


def det_exp(x: float) -> float:
    return float(lib().wo_det_exp(x))


def det_log1m(p: float) -> float:
    return float(lib().wo_det_log1m(p))


def det_u128_to_double(x: int) -> float:
    """The binomial's probability conversion: nearest binary64 to x < 2^128."""
    return float(lib().wo_det_u128_to_double(x & (2 ** 64 - 1), x >> 64))


def det_ldexp(x: float, e: int) -> float:
    return float(lib().wo_det_ldexp(x, e))


def det_lfact(k: int) -> float:
    """log(k!) as the BTRS acceptance test of the OS-ND binomial forms it."""
    return float(lib().wo_det_lfact(k))
