"""Host-side behaviour of the C ABI that needs no GPU: every entry point that
takes a context rejects a NULL one with SSS_ERR_INVALID_ARG before any CUDA
call; the allocation-free doubling rejects a count beyond its fixed capacity
(and NULL pointers) before touching the device; the work-memory sizes are
pure host arithmetic, grow with the input and refuse a text longer than
2^32 - 1; and the binding refuses host tensors for device arguments."""
import ctypes as C

import pytest

import paper_2404_16517_gb300 as sss
from paper_2404_16517_gb300 import _build

INVALID = 1  # SSS_ERR_INVALID_ARG


def _h():
    _build.build()
    return sss.lib()


def _null_args(fn):
    out = []
    for t in fn.argtypes:
        if t in (C.c_uint32, C.c_uint64, C.c_int, C.c_size_t):
            out.append(1)  # a nonzero count: the call must still stop at the context
        else:
            out.append(None)
    return out


CTX_CALLS = ["sss_local_sort", "sss_dist", "sss_dist_prefix", "sss_partition", "sss_lcp_merge", "sss_sort",
             "sss_sort_host", "sss_sort_batch", "sss_suffix_sort", "sss_sync", "sss_set_stream",
             "sss_set_workspace", "sss_set_timing", "sss_reset_stats"]


@pytest.mark.parametrize("name", CTX_CALLS)
def test_null_context_rejected_by_every_entry_point(name):
    fn = getattr(_h(), name)
    assert fn(*_null_args(fn)) == INVALID, name


def test_kernel_stats_and_last_error_without_context():
    h = _h()
    cnt = C.c_uint32(7)
    assert h.sss_kernel_stats(None, None, 0, C.byref(cnt)) == INVALID
    assert h.sss_last_error(None) == b"no context"


def test_noalloc_capacity_and_null_checks_before_the_device():
    h = _h()
    n = sss.NOALLOC_MAX_STRINGS + 1
    assert h.sss_dist_prefix_noalloc(None, 0, None, None, n, None, None, None) == INVALID
    assert h.sss_dist_prefix_noalloc(None, 0, None, None, 5, None, None, None) == INVALID  # NULL arrays
    assert h.sss_dist_prefix_noalloc(None, 0, None, None, 0, None, None, None) == 0  # nothing to do


def test_workspace_sizes_are_host_arithmetic():
    h = _h()
    prm = sss.params()
    sizes = [h.sss_workspace_bytes(n, 100 * n, 16, C.byref(prm)) for n in (1 << 10, 1 << 16, 1 << 22)]
    assert sizes[0] > 0 and sizes[0] <= sizes[1] <= sizes[2]
    assert sizes[2] >= (1 << 22) * 8  # at least the keys of every string
    b = [h.sss_batch_workspace_bytes(n, 64, C.byref(prm)) for n in (1 << 12, 1 << 20)]
    assert 0 < b[0] <= b[1]
    assert h.sss_suffix_workspace_bytes(1 << 20, None) > 0
    assert h.sss_suffix_workspace_bytes(1 << 32, None) == 0  # longer than 2^32 - 1: refused


def test_binding_refuses_host_tensors():
    torch = pytest.importorskip("torch")
    chars = torch.zeros(8, dtype=torch.uint8)
    offs = torch.zeros(2, dtype=torch.int64)
    lens = torch.ones(2, dtype=torch.int32)
    with pytest.raises(ValueError):
        sss.sss_sort(chars, offs, lens, 1)
    with pytest.raises(ValueError):
        sss.sss_dist_prefix(chars, offs, lens)
