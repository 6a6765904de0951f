"""Python binding of libwrs (ctypes; argument marshalling only).

Every function has the name of the C entry point in ``include/wrs.h`` without
the ``wrs_`` prefix and passes its arguments through unchanged: device
pointers and streams are plain integers (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``).  All computation happens in the
CUDA kernels of ``libwrs.so``; there is no CPU fallback: importing this module
without the built library raises.

``AliasTable`` is a small convenience wrapper that owns a table handle and
takes torch tensors (PyTorch is used only for device memory and streams).

With the environment variable ``WRS_CHECK=1`` set before the first import,
the binding loads ``libwrs_check.so`` instead: the same entry points
compiled with bucket write counts and index checks (``wrs_check_build``).
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libwrs_check.so" if os.environ.get("WRS_CHECK") == "1" else "libwrs.so")

OK, EINVAL, ENOMEM, EOVERFLOW, ETIMEOUT, EDEVICE, EINTERNAL = range(7)
U32, F32 = 0, 1
BUCKET_BYTES = 16

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
    )

_lib = ctypes.CDLL(LIB_PATH)


class TableInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("q_lo", ctypes.c_uint64),
        ("q_hi", ctypes.c_uint64),
        ("beta", ctypes.c_int32),
        ("shift", ctypes.c_uint32),
        ("qp", ctypes.c_uint64),
        ("n_light", ctypes.c_uint64),
        ("light_max", ctypes.c_uint32),
        ("status", ctypes.c_int32),
    ]

    @property
    def Q(self) -> int:
        return int(self.q_lo) | (int(self.q_hi) << 64)


_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_I = ctypes.c_int
_TBL = ctypes.c_void_p
_PTBL = ctypes.POINTER(ctypes.c_void_p)

_sig = {
    "wrs_table_create": ([_U64, _PTBL], _I),
    "wrs_table_build": ([_TBL, _P, _U64, _I, _P], _I),
    "wrs_table_build_opts": ([_TBL, _P, _U64, _I, _P, _P], _I),
    "wrs_table_build_psa_plus": ([_TBL, _P, _U64, _I, _P], _I),
    "wrs_table_psa_plus_leftovers": ([_TBL, ctypes.POINTER(ctypes.c_uint64)], _I),
    "wrs_build": ([_P, _U64, _I, _P, _PTBL], _I),
    "wrs_sample": ([_TBL, _U64, _U64, _U64, _P, _P], _I),
    "wrs_table_build_host": ([_TBL, _P, _U64, _I, _P], _I),
    "wrs_sample_host": ([_TBL, _U64, _U64, _U64, _P, _P], _I),
    "wrs_table_status": ([_TBL], _I),
    "wrs_table_info_get": ([_TBL, ctypes.POINTER(TableInfo)], _I),
    "wrs_table_buckets": ([_TBL], _P),
    "wrs_table_download": ([_TBL, _P, _U64], _I),
    "wrs_table_upload": ([_TBL, _P, _U64, _U64, _U64, ctypes.c_int32], _I),
    "wrs_table_set_timing": ([_TBL, _I], _I),
    "wrs_table_stage_ms": ([_TBL, ctypes.POINTER(ctypes.c_float), ctypes.c_uint32], _I),
    "wrs_table_free": ([_TBL], None),
    "wrs_status_str": ([_I], ctypes.c_char_p),
    "wrs_check_build": ([], _I),
    "wrs_table_check_failures": ([_TBL, ctypes.POINTER(ctypes.c_uint64)], _I),
    "wrs_set_wait_limit": ([ctypes.c_uint32], ctypes.c_uint32),
    "wrs_debug_skip_publish": ([ctypes.c_int64], None),
    "wrs_build_noalloc": ([_P, _U64, _I, _P, _P, _P], _I),
    "wrs_batch_offsets": ([ctypes.c_uint32, _P, _P], _I),
    "wrs_batch_create": ([ctypes.c_uint32, _P, _PTBL], _I),
    "wrs_batch_layout": ([_TBL, _P], _I),
    "wrs_batch_buckets": ([_TBL], _P),
    "wrs_batch_build": ([_TBL, _P, _I, _P], _I),
    "wrs_batch_set_samples": ([_TBL, _P, _P], _I),
    "wrs_batch_sample": ([_TBL, _U64, _U64, _P, _P], _I),
    "wrs_batch_status": ([_TBL, _P], _I),
    "wrs_batch_table_info": ([_TBL, ctypes.c_uint32, ctypes.POINTER(TableInfo)], _I),
    "wrs_batch_tune": ([_TBL, _P, _I, _P, ctypes.POINTER(ctypes.c_float)], _I),
    "wrs_batch_groups": ([_TBL, _P], _I),
    "wrs_batch_set_groups": ([_TBL, _P], _I),
    "wrs_batch_download": ([_TBL, _P, _U64], _I),
    "wrs_batch_free": ([_TBL], None),
    "wrs_sample_many": ([_P, ctypes.c_uint32, _U64, _P, _P], _I),
    "wrs_table_device_header": ([_TBL], _P),
    "wrs_batch_device_header": ([_TBL, ctypes.c_uint32], _P),
    "wrs_table2_create": ([_U64, _PTBL], _I),
    "wrs_table2_build": ([_TBL, _P, _U64, _I, _P], _I),
    "wrs_table2_sample": ([_TBL, _U64, _U64, _U64, _P, _P], _I),
    "wrs_table2_status": ([_TBL], _I),
    "wrs_table2_layout": ([_TBL, _P, _P], _I),
    "wrs_table2_download": ([_TBL, _P, _U64, _P, _U64], _I),
    "wrs_table2_free": ([_TBL], None),
    "wrs_table2_sample_os": ([_TBL, _P, _I, _U64, _U64, _U64, _P, _P, _U64, _P, _P], _I),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_sig)


class WrsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_str(code)} ({code})")
        self.code = code


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise WrsError(rc, where)


def status_str(code: int) -> str:
    return _lib.wrs_status_str(code).decode()


# --- thin one-to-one wrappers (return the C status code) -------------------
def table_create(capacity_n: int):
    h = ctypes.c_void_p()
    rc = _lib.wrs_table_create(capacity_n, ctypes.byref(h))
    return rc, h.value


def table_build(t, d_weights: int, n: int, dtype: int, stream: int = 0) -> int:
    return _lib.wrs_table_build(t, d_weights, n, dtype, stream)


ACC_AUTO, ACC_U64, ACC_U128 = range(3)


class BuildOpts(ctypes.Structure):
    """wrs_build_opts: split count (0: the library's choice), tile (0 or
    2048), window (0 or 2048), accumulator mode, flags (0)."""
    _fields_ = [("splits", ctypes.c_uint32), ("tile", ctypes.c_uint32), ("window", ctypes.c_uint32),
                ("acc", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


def table_build_opts(t, d_weights: int, n: int, dtype: int, opts: "BuildOpts | None", stream: int = 0) -> int:
    return _lib.wrs_table_build_opts(t, d_weights, n, dtype, ctypes.byref(opts) if opts is not None else None,
                                     stream)


def table_build_psa_plus(t, d_weights: int, n: int, dtype: int, stream: int = 0) -> int:
    return _lib.wrs_table_build_psa_plus(t, d_weights, n, dtype, stream)


def table_psa_plus_leftovers(t):
    m = ctypes.c_uint64()
    rc = _lib.wrs_table_psa_plus_leftovers(t, ctypes.byref(m))
    return rc, m.value


def build(d_weights: int, n: int, dtype: int, stream: int = 0):
    h = ctypes.c_void_p()
    rc = _lib.wrs_build(d_weights, n, dtype, stream, ctypes.byref(h))
    return rc, h.value


def sample(t, k: int, seed: int, stream_id: int, d_out: int, stream: int = 0) -> int:
    return _lib.wrs_sample(t, k, seed, stream_id, d_out, stream)


def table_build_host(t, h_weights: int, n: int, dtype: int, stream: int = 0) -> int:
    return _lib.wrs_table_build_host(t, h_weights, n, dtype, stream)


def sample_host(t, k: int, seed: int, stream_id: int, h_out: int, stream: int = 0) -> int:
    return _lib.wrs_sample_host(t, k, seed, stream_id, h_out, stream)


def table_status(t) -> int:
    return _lib.wrs_table_status(t)


def table_info_get(t):
    info = TableInfo()
    rc = _lib.wrs_table_info_get(t, ctypes.byref(info))
    return rc, info


def check_build() -> int:
    return _lib.wrs_check_build()


def table_check_failures(t):
    m = ctypes.c_uint64(0)
    rc = _lib.wrs_table_check_failures(t, ctypes.byref(m))
    return rc, m.value


def table_buckets(t) -> int:
    return _lib.wrs_table_buckets(t) or 0


def table_download(t, h_buckets: int, nbytes: int) -> int:
    return _lib.wrs_table_download(t, h_buckets, nbytes)


def table_upload(t, h_buckets: int, n: int, q_lo: int, q_hi: int, beta: int) -> int:
    return _lib.wrs_table_upload(t, h_buckets, n, q_lo, q_hi, beta)


def table_set_timing(t, enable: bool) -> int:
    return _lib.wrs_table_set_timing(t, 1 if enable else 0)


STAGES = ("stats", "stats_combine", "classify", "tilescan", "split", "sweep")


def table_stage_ms(t, count: int = 5):
    buf = (ctypes.c_float * count)()
    rc = _lib.wrs_table_stage_ms(t, buf, count)
    return rc, [float(x) for x in buf]


def table_free(t) -> None:
    _lib.wrs_table_free(t)


def set_wait_limit(polls: int) -> int:
    return _lib.wrs_set_wait_limit(polls)


def debug_skip_publish(tile: int) -> None:
    _lib.wrs_debug_skip_publish(tile)


NOALLOC_MAX_N = 1 << 22
DEVICE_HEADER_BYTES = 128


def build_noalloc(d_weights: int, n: int, dtype: int, d_buckets: int, d_header: int, stream: int = 0) -> int:
    """wrs_build_noalloc: build into caller-owned buckets and header using the
    library's static scratch (no allocation)."""
    return _lib.wrs_build_noalloc(d_weights, n, dtype, d_buckets, d_header, stream)


BATCH_CLASSES = 5


def _u64_array(values):
    vals = [int(v) for v in values]
    return (ctypes.c_uint64 * max(1, len(vals)))(*vals)


def batch_offsets(sizes):
    """wrs_batch_offsets: (rc, word offsets of the tables, total words last)."""
    arr = _u64_array(sizes)
    out = (ctypes.c_uint64 * (len(sizes) + 1))()
    rc = _lib.wrs_batch_offsets(len(sizes), arr, out)
    return rc, [int(x) for x in out]


def batch_create(sizes):
    h = ctypes.c_void_p()
    rc = _lib.wrs_batch_create(len(sizes), _u64_array(sizes), ctypes.byref(h))
    return rc, h.value


def batch_build(b, d_weights: int, dtype: int, stream: int = 0) -> int:
    return _lib.wrs_batch_build(b, d_weights, dtype, stream)


def batch_set_samples(b, ks):
    out = (ctypes.c_uint64 * (len(ks) + 1))()
    rc = _lib.wrs_batch_set_samples(b, _u64_array(ks), out)
    return rc, [int(x) for x in out]


def batch_sample(b, seed: int, stream_id: int, d_out: int, stream: int = 0) -> int:
    return _lib.wrs_batch_sample(b, seed, stream_id, d_out, stream)


def batch_status(b, ntables: int):
    st = (ctypes.c_int32 * ntables)()
    rc = _lib.wrs_batch_status(b, st)
    return rc, [int(x) for x in st]


def batch_table_info(b, table: int):
    info = TableInfo()
    rc = _lib.wrs_batch_table_info(b, table, ctypes.byref(info))
    return rc, info


def batch_tune(b, d_weights: int, dtype: int, stream: int = 0):
    ms = ctypes.c_float()
    rc = _lib.wrs_batch_tune(b, d_weights, dtype, stream, ctypes.byref(ms))
    return rc, float(ms.value)


def batch_groups(b):
    g = (ctypes.c_uint32 * BATCH_CLASSES)()
    rc = _lib.wrs_batch_groups(b, g)
    return rc, [int(x) for x in g]


def batch_set_groups(b, groups) -> int:
    g = (ctypes.c_uint32 * BATCH_CLASSES)(*[int(x) for x in groups])
    return _lib.wrs_batch_set_groups(b, g)


def batch_buckets(b) -> int:
    return _lib.wrs_batch_buckets(b) or 0


def batch_download(b, h_buckets: int, nbytes: int) -> int:
    return _lib.wrs_batch_download(b, h_buckets, nbytes)


def batch_free(b) -> None:
    _lib.wrs_batch_free(b)


SAMPLE_TASK_BYTES = 64  # wrs_sample_task: 8 little-endian 64-bit words


def sample_many(d_tasks: int, ntasks: int, total_k: int, d_out: int, stream: int = 0) -> int:
    return _lib.wrs_sample_many(d_tasks, ntasks, total_k, d_out, stream)


def table_device_header(t) -> int:
    return _lib.wrs_table_device_header(t) or 0


def batch_device_header(b, table: int) -> int:
    return _lib.wrs_batch_device_header(b, table) or 0


# --- convenience wrapper over torch tensors --------------------------------
def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.float32:
        return F32
    if t.dtype in (torch.uint32, torch.int32):
        return U32
    raise TypeError(f"weights must be float32 or uint32/int32 words, got {t.dtype}")


def _require_cuda(x, what: str, min_numel: int = 0, itemsize: int | None = None) -> None:
    """Refuse, before any launch, what the kernels must not see: a host
    tensor (its pointer is not device memory), a strided view, too few
    elements, or elements of the wrong size."""
    if not x.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if x.numel() < min_numel:
        raise ValueError(f"{what} holds {x.numel()} elements, {min_numel} needed")
    if itemsize is not None and x.element_size() != itemsize:
        raise ValueError(f"{what} must have {itemsize}-byte elements, not {x.element_size()}")


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class AliasTable:
    """Owns one device-resident alias table (``wrs_table``)."""

    def __init__(self, capacity_n: int):
        rc, h = table_create(capacity_n)
        _check(rc, "wrs_table_create")
        self.handle = h
        self.capacity = capacity_n
        self.n = 0

    def build(self, weights, stream=None) -> "AliasTable":
        """weights: contiguous CUDA tensor of float32 or uint32/int32 words."""
        _require_cuda(weights, "weights")
        n = weights.numel()
        _check(table_build(self.handle, weights.data_ptr(), n, _dtype_code(weights), _stream_handle(stream)),
               "wrs_table_build")
        self.n = n
        return self

    def build_opts(self, weights, splits: int = 0, acc: int = 0, tile: int = 0, window: int = 0,
                   stream=None) -> "AliasTable":
        """wrs_table_build_opts: the same table for every split count and
        accumulator mode; they choose how the work is cut."""
        _require_cuda(weights, "weights")
        n = weights.numel()
        o = BuildOpts(splits=splits, tile=tile, window=window, acc=acc, flags=0)
        _check(table_build_opts(self.handle, weights.data_ptr(), n, _dtype_code(weights), o, _stream_handle(stream)),
               "wrs_table_build_opts")
        self.n = n
        return self

    def build_psa_plus(self, weights, stream=None) -> "AliasTable":
        """PSA+ build (per-tile greedy pass, then PSA on the leftovers)."""
        _require_cuda(weights, "weights")
        n = weights.numel()
        _check(table_build_psa_plus(self.handle, weights.data_ptr(), n, _dtype_code(weights),
                                    _stream_handle(stream)), "wrs_table_build_psa_plus")
        self.n = n
        return self

    def psa_plus_leftovers(self) -> int:
        rc, m = table_psa_plus_leftovers(self.handle)
        _check(rc, "wrs_table_psa_plus_leftovers")
        return m

    def sample(self, k: int, seed: int, stream_id: int = 0, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(k, dtype=torch.int32, device="cuda")
        _require_cuda(out, "out", k, 4)
        _check(sample(self.handle, k, seed, stream_id, out.data_ptr(), _stream_handle(stream)), "wrs_sample")
        return out

    def status(self) -> int:
        return table_status(self.handle)

    def set_timing(self, enable: bool = True) -> None:
        _check(table_set_timing(self.handle, enable), "wrs_table_set_timing")

    def stage_ms(self) -> dict:
        rc, ms = table_stage_ms(self.handle, len(STAGES))
        _check(rc, "wrs_table_stage_ms")
        return dict(zip(STAGES, ms))

    def info(self) -> TableInfo:
        rc, info = table_info_get(self.handle)
        _check(rc, "wrs_table_info_get")
        return info

    def check_failures(self) -> int:
        rc, m = table_check_failures(self.handle)
        _check(rc, "wrs_table_check_failures")
        return m

    def download(self):
        import numpy as np

        buf = np.empty(self.n * 2, dtype=np.uint64)
        _check(table_download(self.handle, buf.ctypes.data, buf.nbytes), "wrs_table_download")
        words = buf.view(np.uint32).reshape(self.n, 4)
        thr = buf.reshape(self.n, 2)[:, 0].copy()
        alias = words[:, 2].copy()
        return thr, alias, words[:, 3].copy()

    def free(self) -> None:
        if self.handle:
            table_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class AliasBatch:
    """Owns a batch of independent device-resident alias tables (``wrs_batch``).

    ``weights`` buffers are laid out by ``offsets`` (table t at word
    ``offsets[t]``); ``pack`` builds such a buffer from a list of tensors."""

    def __init__(self, sizes):
        self.sizes = [int(x) for x in sizes]
        rc, h = batch_create(self.sizes)
        _check(rc, "wrs_batch_create")
        self.handle = h
        rc, self.offsets = batch_offsets(self.sizes)
        _check(rc, "wrs_batch_offsets")
        self.k_offsets = None

    @property
    def ntables(self) -> int:
        return len(self.sizes)

    def pack(self, tensors, dtype=None):
        """One CUDA weight buffer holding the given per-table tensors at their offsets."""
        import torch

        dtype = dtype or tensors[0].dtype
        buf = torch.zeros(self.offsets[-1], dtype=dtype, device="cuda")
        for t, x in enumerate(tensors):
            if x.numel() != self.sizes[t]:
                raise ValueError(f"table {t} has {self.sizes[t]} weights, got {x.numel()}")
            buf[self.offsets[t]:self.offsets[t] + self.sizes[t]].copy_(x.reshape(-1))
        return buf

    def build(self, weights, stream=None) -> "AliasBatch":
        _require_cuda(weights, "weights", self.offsets[-1])
        _check(batch_build(self.handle, weights.data_ptr(), _dtype_code(weights), _stream_handle(stream)),
               "wrs_batch_build")
        return self

    def set_samples(self, ks) -> list:
        if len(ks) != self.ntables:
            raise ValueError(f"{self.ntables} sample counts needed, got {len(ks)}")
        rc, self.k_offsets = batch_set_samples(self.handle, ks)
        _check(rc, "wrs_batch_set_samples")
        return self.k_offsets

    def sample(self, seed: int, stream_id: int = 0, out=None, stream=None):
        import torch

        total = self.k_offsets[-1] if self.k_offsets else 0
        if out is None:
            out = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        _require_cuda(out, "out", total, 4)
        _check(batch_sample(self.handle, seed, stream_id, out.data_ptr(), _stream_handle(stream)),
               "wrs_batch_sample")
        return out

    def status(self):
        return batch_status(self.handle, self.ntables)

    def info(self, table: int) -> TableInfo:
        rc, info = batch_table_info(self.handle, table)
        _check(rc, "wrs_batch_table_info")
        return info

    def tune(self, weights, stream=None) -> float:
        rc, ms = batch_tune(self.handle, weights.data_ptr(), _dtype_code(weights), _stream_handle(stream))
        _check(rc, "wrs_batch_tune")
        return ms

    def groups(self):
        rc, g = batch_groups(self.handle)
        _check(rc, "wrs_batch_groups")
        return g

    def set_groups(self, groups) -> None:
        _check(batch_set_groups(self.handle, groups), "wrs_batch_set_groups")

    def download(self):
        """(thr, alias, reserved) numpy arrays over all buckets (table t at offsets[t])."""
        import numpy as np

        total = self.offsets[-1]
        buf = np.empty(total * 2, dtype=np.uint64)
        _check(batch_download(self.handle, buf.ctypes.data, buf.nbytes), "wrs_batch_download")
        words = buf.view(np.uint32).reshape(total, 4)
        return buf.reshape(total, 2)[:, 0].copy(), words[:, 2].copy(), words[:, 3].copy()

    def free(self) -> None:
        if self.handle:
            batch_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


TABLE2_GROUP = 2048
TABLE2_MAX_LEVELS = 4


def table2_create(capacity_n: int):
    h = ctypes.c_void_p()
    rc = _lib.wrs_table2_create(capacity_n, ctypes.byref(h))
    return rc, h.value


def table2_build(t, d_weights: int, n: int, dtype: int, stream: int = 0) -> int:
    return _lib.wrs_table2_build(t, d_weights, n, dtype, stream)


def table2_sample(t, k: int, seed: int, stream_id: int, d_out: int, stream: int = 0) -> int:
    return _lib.wrs_table2_sample(t, k, seed, stream_id, d_out, stream)


def table2_status(t) -> int:
    return _lib.wrs_table2_status(t)


def table2_layout(t):
    L = ctypes.c_uint32()
    sizes = (ctypes.c_uint64 * TABLE2_MAX_LEVELS)()
    rc = _lib.wrs_table2_layout(t, ctypes.byref(L), sizes)
    return rc, [int(sizes[i]) for i in range(L.value)]


def table2_download(t, h_buckets: int, bucket_bytes: int, h_groups: int, group_bytes: int) -> int:
    return _lib.wrs_table2_download(t, h_buckets, bucket_bytes, h_groups, group_bytes)


def table2_free(t) -> None:
    _lib.wrs_table2_free(t)


def table2_sample_os(t, d_weights: int, dtype: int, k: int, seed: int, stream_id: int, d_items: int,
                     d_counts: int, capacity: int, d_npairs: int, stream: int = 0) -> int:
    return _lib.wrs_table2_sample_os(t, d_weights, dtype, k, seed, stream_id, d_items, d_counts, capacity,
                                     d_npairs, stream)


class AliasTable2:
    """Owns one two-level ("2lvl-sweep") table (``wrs_table2``)."""

    def __init__(self, capacity_n: int):
        rc, h = table2_create(capacity_n)
        _check(rc, "wrs_table2_create")
        self.handle = h
        self.capacity = capacity_n
        self.n = 0

    def build(self, weights, stream=None) -> "AliasTable2":
        _require_cuda(weights, "weights")
        n = weights.numel()
        _check(table2_build(self.handle, weights.data_ptr(), n, _dtype_code(weights), _stream_handle(stream)),
               "wrs_table2_build")
        self.n = n
        return self

    def sample(self, k: int, seed: int, stream_id: int = 0, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(max(k, 1), dtype=torch.int32, device="cuda")
        _require_cuda(out, "out", k, 4)
        _check(table2_sample(self.handle, k, seed, stream_id, out.data_ptr(), _stream_handle(stream)),
               "wrs_table2_sample")
        return out

    def status(self) -> int:
        return table2_status(self.handle)

    def sample_os(self, weights, k: int, seed: int, stream_id: int = 0, capacity: int | None = None,
                  stream=None):
        """OS-ND sampling: (items, counts) CUDA tensors of the pairs drawn
        (synchronises to read their number).  ``weights`` are the words the
        table was built from."""
        import torch

        _require_cuda(weights, "weights", self.n)
        if capacity is None:
            capacity = min(k, self.n + 128 * (self.n // TABLE2_GROUP + 1)) + 1
        items = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
        counts = torch.empty(max(capacity, 1), dtype=torch.int64, device="cuda")
        npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
        _check(table2_sample_os(self.handle, weights.data_ptr(), _dtype_code(weights), k, seed, stream_id,
                                items.data_ptr(), counts.data_ptr(), capacity, npairs.data_ptr(),
                                _stream_handle(stream)), "wrs_table2_sample_os")
        m = int(npairs.item())
        if m > capacity:
            raise WrsError(ENOMEM, f"wrs_table2_sample_os: {m} pairs exceed the capacity {capacity}")
        return items[:m], counts[:m]

    def levels(self):
        rc, sizes = table2_layout(self.handle)
        _check(rc, "wrs_table2_layout")
        return sizes

    def download(self):
        """(thr, alias) over all levels (level 0 first) and per group (qp, shift, members)."""
        import numpy as np

        sizes = self.levels()
        nb = sum(sizes)
        ng = sum((m + TABLE2_GROUP - 1) // TABLE2_GROUP for m in sizes)
        buf = np.empty(nb * 2, dtype=np.uint64)
        grp = np.empty(ng * 2, dtype=np.uint64)
        _check(table2_download(self.handle, buf.ctypes.data, buf.nbytes, grp.ctypes.data, grp.nbytes),
               "wrs_table2_download")
        words = buf.view(np.uint32).reshape(nb, 4)
        gw = grp.view(np.uint32).reshape(ng, 4)
        return (buf.reshape(nb, 2)[:, 0].copy(), words[:, 2].copy(), words[:, 3].copy(),
                grp.reshape(ng, 2)[:, 0].copy(), gw[:, 2].copy(), gw[:, 3].copy())

    def free(self) -> None:
        if self.handle:
            table2_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
