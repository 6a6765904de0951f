"""The C-ABI library loads, exports every entry point include/wrs.h declares,
and rejects bad arguments before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wrs():
    import __graft_entry__ as g

    g.build()
    from paper_1903_00227_gb300 import wrs as W

    return W


def declared_functions():
    text = open(os.path.join(ROOT, "include", "wrs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wrs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(wrs):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(wrs.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(wrs.EXPORTED) == names


def test_check_build_exports_the_same_symbols(wrs):
    """libwrs_check.so (WRS_CHECK=1) has every entry point of the standard
    library and says which build it is; the standard library says 0."""
    names = declared_functions()
    check = ctypes.CDLL(os.path.join(os.path.dirname(wrs.LIB_PATH), "libwrs_check.so"))
    for name in names:
        assert hasattr(check, name), name
    check.wrs_check_build.restype = ctypes.c_int
    assert check.wrs_check_build() == 1
    assert wrs.check_build() == (1 if wrs.LIB_PATH.endswith("libwrs_check.so") else 0)
    assert wrs.table_check_failures(None)[0] == wrs.EINVAL


def test_argument_errors_need_no_gpu(wrs):
    rc, h = wrs.table_create(0)
    assert rc == wrs.EINVAL and h is None
    rc, h = wrs.table_create(1 << 32)
    assert rc == wrs.EINVAL
    assert wrs.table_build(None, 0, 10, wrs.U32, 0) == wrs.EINVAL
    assert wrs.table_build_opts(None, 0, 10, wrs.U32, wrs.BuildOpts(), 0) == wrs.EINVAL
    assert wrs.table_build_opts(None, 16, 10, wrs.U32, None, 0) == wrs.EINVAL
    assert wrs.sample(None, 10, 1, 0, 0, 0) == wrs.EINVAL
    assert wrs.table_status(None) == wrs.EINVAL
    assert wrs.table_download(None, 0, 0) == wrs.EINVAL
    assert wrs.table_buckets(None) == 0
    wrs.table_free(None)


def test_status_strings(wrs):
    seen = {wrs.status_str(c) for c in range(7)}
    assert len(seen) == 7
    assert wrs.status_str(99) == "unknown status"


def test_bucket_layout_matches_header():
    text = open(os.path.join(ROOT, "include", "wrs.h")).read()
    assert re.search(r"uint64_t thr;\s*uint32_t alias;\s*uint32_t reserved;", text)


def test_batch_offsets_host_only(wrs):
    sizes = [1, 2, 3, 4, 5, 2048, 2049, 7]
    rc, off = wrs.batch_offsets(sizes)
    assert rc == wrs.OK and len(off) == len(sizes) + 1 and off[0] == 0
    for t, n in enumerate(sizes):
        assert off[t] % 4 == 0, "each table starts 16-byte aligned"
        assert off[t] + n <= off[t + 1] < off[t] + n + 4, "tables are packed in order"
    assert wrs.batch_offsets([3, 0])[0] == wrs.EINVAL
    assert wrs.batch_offsets([1 << 32])[0] == wrs.EINVAL
    assert wrs.batch_create([])[0] == wrs.EINVAL
    assert wrs.batch_build(None, 0, wrs.F32, 0) == wrs.EINVAL
    assert wrs.batch_sample(None, 1, 0, 0, 0) == wrs.EINVAL
    assert wrs.batch_buckets(None) == 0
    wrs.batch_free(None)


def test_every_entry_point_rejects_null_handles_without_a_gpu(wrs):
    """Null handles and missing buffers are refused with WRS_EINVAL before any
    CUDA call, for every entry point that takes a table, a batch or a task
    list (the library is loaded on a machine with no GPU)."""
    lib = wrs._lib  # argument and result types as the binding declares them
    E = wrs.EINVAL
    # single tables
    assert wrs.table_build_host(None, 0, 10, wrs.F32, 0) == E
    assert wrs.sample_host(None, 10, 1, 0, 0, 0) == E
    assert wrs.table_upload(None, 0, 10, 1, 0, 0) == E
    assert wrs.table_set_timing(None, True) == E
    assert wrs.table_build_psa_plus(None, 0, 10, wrs.F32, 0) == E
    assert wrs.table_psa_plus_leftovers(None)[0] == E
    assert lib.wrs_table_info_get(None, None) == E
    assert lib.wrs_table_device_header(None) is None
    # the allocation-free build: missing buffers, sizes past its scratch
    assert wrs.build_noalloc(0, 10, wrs.F32, 0, 0, 0) == E
    assert wrs.build_noalloc(16, 0, wrs.F32, 16, 16, 0) == E
    # batches
    assert lib.wrs_batch_create(0, None, None) == E
    assert wrs.batch_build(None, 16, wrs.F32, 0) == E
    assert wrs.batch_sample(None, 1, 0, 16, 0) == E
    assert wrs.batch_download(None, 16, 16) == E
    assert lib.wrs_batch_layout(None, None) == E
    assert lib.wrs_batch_groups(None, None) == E
    assert lib.wrs_batch_set_groups(None, None) == E
    assert lib.wrs_batch_status(None, None) == E
    assert lib.wrs_batch_buckets(None) is None
    assert lib.wrs_batch_device_header(None, 0) is None
    wrs.batch_free(None)
    # many sample requests: nothing to draw is fine, a missing task list is not
    assert wrs.sample_many(0, 0, 0, 0, 0) == wrs.OK
    assert wrs.sample_many(0, 1, 10, 16, 0) == E
    assert wrs.sample_many(8, 1, 10, 16, 0) == E  # task list not 16-byte aligned
    # two-level tables and OS-ND
    assert wrs.table2_build(None, 16, 10, wrs.F32, 0) == E
    assert wrs.table2_sample(None, 10, 1, 0, 16, 0) == E
    assert wrs.table2_status(None) == E
    assert wrs.table2_download(None, 16, 16, 16, 16) == E
    assert lib.wrs_table2_layout(None, None, None) == E
    assert lib.wrs_table2_sample_os(None, None, 1, 10, 1, 0, None, None, 0, None, None) == E
    wrs.table2_free(None)


def test_binding_refuses_what_the_kernels_must_not_see():
    """Host tensors, strided views, short outputs and wrong element sizes are
    refused before any launch (explicit checks that stay under python -O)."""
    import torch

    from paper_1903_00227_gb300 import wrs

    with pytest.raises(ValueError, match="CUDA tensor"):
        wrs._require_cuda(torch.zeros(8), "weights")
    with pytest.raises(ValueError, match="CUDA tensor"):
        wrs._require_cuda(torch.zeros(8, dtype=torch.int32), "out", 8, 4)
    with pytest.raises(TypeError):
        wrs._dtype_code(torch.zeros(4, dtype=torch.float64))


class _DeviceLike:
    """Stands in for a CUDA tensor's metadata (no device needed)."""

    is_cuda = True

    def __init__(self, numel, itemsize=4, contiguous=True):
        self._n, self._s, self._c = numel, itemsize, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def element_size(self):
        return self._s


def test_binding_checks_layout_size_and_element_size():
    from paper_1903_00227_gb300 import wrs

    wrs._require_cuda(_DeviceLike(8), "out", 8, 4)  # accepted
    with pytest.raises(ValueError, match="contiguous"):
        wrs._require_cuda(_DeviceLike(8, contiguous=False), "weights")
    with pytest.raises(ValueError, match="7 elements, 8 needed"):
        wrs._require_cuda(_DeviceLike(7), "out", 8, 4)
    with pytest.raises(ValueError, match="4-byte elements"):
        wrs._require_cuda(_DeviceLike(8, itemsize=8), "out", 8, 4)
