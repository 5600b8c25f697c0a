"""GB300 string sorter: thin Python binding over the C ABI of ``libsss.so``.

The functions here only marshal arguments (torch CUDA tensors -> device
pointers, the current torch stream -> the context stream) and call the C entry
points of the same names declared in ``include/sss.h``; every step of the sort
runs in the library's CUDA kernels.  If the library is not built the calls raise
``RuntimeError``: there is no CPU fallback.

String sets are passed as three tensors on one CUDA device:
``chars`` (uint8, N), ``offs`` (int64 holding uint64 offsets, n) and ``lens``
(int32 holding uint32 lengths, n); outputs are int32 tensors holding uint32
values.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsss.so")

SSS_FLAG_MS = 0x1
SSS_FLAG_CHECKED = 0x2
SSS_FLAG_NO_LOCAL_LCP_SKIP = 0x4
SSS_FLAG_DEDUPE_SORT = 0x8
SSS_FLAG_MERGE_TREE = 0x10
SSS_FLAG_CHAR_SAMPLING = 0x20
SSS_FLAG_GRAPH = 0x40
SSS_FLAG_NO_CTA_ROUNDS = 0x80
SSS_KMAX_AUTO = 0xFFFFFFFF
SSS_MAX_KERNELS = 128

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "device wait timed out",
          5: "input validation failed on the device", 6: "not implemented", 7: "workspace too small"}


class SssError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sss status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class sss_params(C.Structure):
    _fields_ = [("kmin", C.c_uint32), ("kmax", C.c_uint32), ("v", C.c_uint32), ("flags", C.c_uint32),
                ("hash_seed", C.c_uint64), ("cta_cap", C.c_uint32), ("merge_ms", C.c_uint32),
                ("direct_cap", C.c_uint32), ("bucket_target", C.c_uint32), ("warp_cap", C.c_uint32),
                ("reserved", C.c_uint32 * 1)]

TUNING_FIELDS = ("cta_cap", "merge_ms", "direct_cap", "bucket_target", "warp_cap")


class sss_instance(C.Structure):
    _fields_ = [("first", C.c_uint64), ("n", C.c_uint32), ("p", C.c_uint32)]


class sss_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_uint64), ("total_ms", C.c_double), ("timed", C.c_uint64)]


_lib_handle = None
_lib_lock = threading.Lock()


def lib():
    """Load libsss.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    with _lib_lock:
        if _lib_handle is not None:
            return _lib_handle
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        h = C.CDLL(LIB_PATH)
        vp, u32, u64, st = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        P = C.POINTER(sss_params)
        sigs = {
            "sss_params_default": (None, [P]),
            "sss_create": (st, [C.POINTER(C.c_void_p), C.c_int, vp]),
            "sss_destroy": (st, [vp]),
            "sss_set_stream": (st, [vp, vp]),
            "sss_set_workspace": (st, [vp, vp, C.c_size_t]),
            "sss_workspace_bytes": (C.c_size_t, [u32, u64, u32, P]),
            "sss_batch_workspace_bytes": (C.c_size_t, [u32, u32, P]),
            "sss_suffix_workspace_bytes": (C.c_size_t, [u64, P]),
            "sss_suffix_sort": (st, [vp, vp, u64, u32, P, vp, vp]),
            "sss_sync": (st, [vp]),
            "sss_status_string": (C.c_char_p, [st]),
            "sss_last_error": (C.c_char_p, [vp]),
            "sss_local_sort": (st, [vp, vp, u64, vp, vp, u32, u32, P, vp, vp]),
            "sss_dist": (st, [vp, vp, u32, vp, vp, vp]),
            "sss_dist_prefix": (st, [vp, vp, u64, vp, vp, u32, vp, vp, u32, P, vp]),
            "sss_partition": (st, [vp, vp, u64, vp, vp, vp, vp, u32, u32, P, vp, vp]),
            "sss_lcp_merge": (st, [vp, vp, u64, vp, vp, vp, vp, vp, u32, u32, P, vp, vp]),
            "sss_sort": (st, [vp, vp, u64, vp, vp, u32, u32, P, vp, vp, vp, vp]),
            "sss_sort_host": (st, [vp, vp, u64, vp, vp, u32, u32, P, vp, vp, vp, vp, vp, vp, vp]),
            "sss_dist_prefix_noalloc": (st, [vp, u64, vp, vp, u32, P, vp, vp]),
            "sss_sort_batch": (st, [vp, vp, u64, vp, vp, u32, C.POINTER(sss_instance), u32, P, vp, vp, vp]),
            "sss_set_timing": (st, [vp, C.c_int, C.c_char_p]),
            "sss_kernel_stats": (st, [vp, C.POINTER(sss_kernel_stat), u32, C.POINTER(u32)]),
            "sss_reset_stats": (st, [vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib_handle = h
    return _lib_handle


def exported_symbols() -> list[str]:
    """Names of the sss_* functions this binding binds (all declared in sss.h)."""
    return ["sss_params_default", "sss_create", "sss_destroy", "sss_set_stream", "sss_set_workspace",
            "sss_workspace_bytes", "sss_sync", "sss_status_string", "sss_last_error", "sss_local_sort",
            "sss_dist", "sss_dist_prefix", "sss_partition", "sss_lcp_merge", "sss_sort", "sss_set_timing",
            "sss_kernel_stats", "sss_reset_stats", "sss_dist_prefix_noalloc", "sss_sort_batch", "sss_sort_host",
            "sss_batch_workspace_bytes", "sss_suffix_workspace_bytes", "sss_suffix_sort"]


def params(kmin: int = 0, kmax: int = SSS_KMAX_AUTO, v: int = 2, flags: int = 0, hash_seed: int = 0,
           cta_cap: int = 0, merge_ms: int = 0, direct_cap: int = 0, bucket_target: int = 0,
           warp_cap: int = 0) -> sss_params:
    """sss_params; the tuning knobs (0 = default) change speed, never results."""
    p = sss_params()
    lib().sss_params_default(C.byref(p))
    p.kmin, p.kmax, p.v, p.flags, p.hash_seed, p.cta_cap = kmin, kmax, v, flags, hash_seed, cta_cap
    p.merge_ms, p.direct_cap, p.bucket_target, p.warp_cap = merge_ms, direct_cap, bucket_target, warp_cap
    return p


class Context:
    """One sss_ctx bound to a CUDA device; enqueues on torch's current stream."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = C.c_void_p()
        self._check(lib().sss_create(C.byref(h), self.device, C.c_void_p(self._stream())), None)
        self.h = h

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _check(self, status: int, h=None):
        if status != 0:
            msg = lib().sss_last_error(h if h is not None else getattr(self, "h", None))
            raise SssError(status, (msg or b"").decode())

    def bind_stream(self):
        self._check(lib().sss_set_stream(self.h, C.c_void_p(self._stream())), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().sss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        self._check(lib().sss_sync(self.h), self.h)

    def set_workspace(self, t: torch.Tensor | None):
        if t is None:
            self._check(lib().sss_set_workspace(self.h, None, 0), self.h)
        else:
            self._check(lib().sss_set_workspace(self.h, C.c_void_p(t.data_ptr()), t.numel() * t.element_size()),
                        self.h)

    def set_timing(self, enable: bool, name_filter: str = ""):
        self._check(lib().sss_set_timing(self.h, 1 if enable else 0, name_filter.encode()), self.h)

    def kernel_stats(self) -> dict:
        arr = (sss_kernel_stat * SSS_MAX_KERNELS)()
        cnt = C.c_uint32()
        self._check(lib().sss_kernel_stats(self.h, arr, SSS_MAX_KERNELS, C.byref(cnt)), self.h)
        return {arr[i].name.decode(): dict(launches=int(arr[i].launches), total_ms=float(arr[i].total_ms),
                                           timed=int(arr[i].timed)) for i in range(cnt.value)}

    def reset_stats(self):
        self._check(lib().sss_reset_stats(self.h), self.h)


_ctx_cache: dict[int, Context] = {}


def context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    c = _ctx_cache.get(device)
    if c is None:
        c = Context(device)
        _ctx_cache[device] = c
    c.bind_stream()
    return c


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_strings(chars, offs, lens):
    for t, dt, name in ((chars, torch.uint8, "chars"), (offs, torch.int64, "offs"), (lens, torch.int32, "lens")):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {dt}")
    if offs.numel() != lens.numel():
        raise ValueError("offs and lens must have the same length")


# When set (the test suite sets SSS_FILL_OUTPUTS=1), every output tensor is
# filled with 0xFFFFFFFF on the call's stream before the library writes it, so a
# kernel that leaves a position unwritten cannot pass a comparison on memory the
# caching allocator handed back still holding an earlier, correct result.
FILL_OUTPUTS = os.environ.get("SSS_FILL_OUTPUTS", "") == "1"


def _sentinel(t, n):
    if FILL_OUTPUTS and t is not None and n > 0:
        t[:n].fill_(-1)
    return t


def _out(t, n, device):
    if t is None:
        return _sentinel(torch.empty(n, dtype=torch.int32, device=device), n)
    if not t.is_cuda or t.dtype != torch.int32 or t.numel() < n or not t.is_contiguous():
        raise ValueError("output tensors must be contiguous int32 CUDA tensors of length >= n")
    return _sentinel(t, n)


def sss_local_sort(chars, offs, lens, p: int = 1, prm: sss_params | None = None, out_run_perm=None,
                   out_run_lcp=None, ctx: Context | None = None):
    """Stage A: sorted runs and LCP arrays of p partitions."""
    _check_strings(chars, offs, lens)
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    rp, rl = _out(out_run_perm, n, chars.device), _out(out_run_lcp, n, chars.device)
    prm = prm or params()
    ctx._check(lib().sss_local_sort(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), n, p, C.byref(prm),
                                    _ptr(rp), _ptr(rl)), ctx.h)
    return rp, rl


def sss_dist(lens, perm, lcp, out_dist=None, ctx: Context | None = None):
    """Stage A6: exact distinguishing prefixes from a global order."""
    ctx = ctx or context(lens.device.index)
    n = lens.numel()
    d = _out(out_dist, n, lens.device)
    ctx._check(lib().sss_dist(ctx.h, _ptr(lens), n, _ptr(perm), _ptr(lcp), _ptr(d)), ctx.h)
    return d


def sss_dist_prefix(chars, offs, lens, run_perm=None, run_lcp=None, p: int = 1, prm: sss_params | None = None,
                    out_approx=None, ctx: Context | None = None):
    """Stage B: approximate distinguishing prefixes by prefix doubling."""
    _check_strings(chars, offs, lens)
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    a = _out(out_approx, n, chars.device)
    prm = prm or params()
    ctx._check(lib().sss_dist_prefix(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), n, _ptr(run_perm),
                                     _ptr(run_lcp), p, C.byref(prm), _ptr(a)), ctx.h)
    return a


def sss_partition(chars, offs, lens, run_perm, p: int, trunc=None, prm: sss_params | None = None,
                  ctx: Context | None = None):
    """Stage C: splitters (p-1) and bucket bounds (p x (p+1))."""
    _check_strings(chars, offs, lens)
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    spl = _sentinel(torch.empty(max(p - 1, 1), dtype=torch.int32, device=chars.device), max(p - 1, 1))
    bnd = _sentinel(torch.empty(p * (p + 1), dtype=torch.int32, device=chars.device), p * (p + 1))
    prm = prm or params()
    ctx._check(lib().sss_partition(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), _ptr(trunc),
                                   _ptr(run_perm), n, p, C.byref(prm), _ptr(spl), _ptr(bnd)), ctx.h)
    return spl[:p - 1], bnd.view(p, p + 1)


def sss_lcp_merge(chars, offs, lens, run_perm, run_lcp, p: int, trunc=None, prm: sss_params | None = None,
                  out_perm=None, out_lcp=None, ctx: Context | None = None):
    """Stage D: LCP-compressed exchange and LCP merge of p sorted runs."""
    _check_strings(chars, offs, lens)
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    op, ol = _out(out_perm, n, chars.device), _out(out_lcp, n, chars.device)
    prm = prm or params()
    ctx._check(lib().sss_lcp_merge(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), _ptr(trunc),
                                   _ptr(run_perm), _ptr(run_lcp), n, p, C.byref(prm), _ptr(op), _ptr(ol)), ctx.h)
    return op, ol


def sss_sort(chars, offs, lens, p: int = 1, prm: sss_params | None = None, out_perm=None, out_lcp=None,
             want_dist: bool = False, want_approx: bool = False, out_dist=None, out_approx=None,
             ctx: Context | None = None):
    """The whole path: returns (perm, lcp, dist or None, approx or None)."""
    _check_strings(chars, offs, lens)
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    op, ol = _out(out_perm, n, chars.device), _out(out_lcp, n, chars.device)
    d = _out(out_dist, n, chars.device) if (want_dist or out_dist is not None) else None
    a = _out(out_approx, n, chars.device) if (want_approx or out_approx is not None) else None
    prm = prm or params()
    ctx._check(lib().sss_sort(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), n, p, C.byref(prm),
                              _ptr(op), _ptr(ol), _ptr(d), _ptr(a)), ctx.h)
    return op, ol, d, a


def sss_sort_host(h_chars, h_offs, h_lens, p: int, d_chars, d_offs, d_lens, prm: sss_params | None = None,
                  out_perm=None, out_lcp=None, h_out_perm=None, h_out_lcp=None, ctx: Context | None = None):
    """The whole path for a string set in host memory (CPU tensors, pinned for
    full copy speed), the upload overlapped with the local sorts.  d_chars/d_offs/
    d_lens are device buffers of the same sizes that the call fills; h_out_perm/
    h_out_lcp (CPU int32 tensors or None) receive copies of the outputs once the
    stream is synchronised.  Returns the device (perm, lcp)."""
    for t, dt, name in ((h_chars, torch.uint8, "h_chars"), (h_offs, torch.int64, "h_offs"),
                        (h_lens, torch.int32, "h_lens")):
        if t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor of dtype {dt}")
    _check_strings(d_chars, d_offs, d_lens)
    n = h_lens.numel()
    if h_offs.numel() != n or d_lens.numel() < n or d_offs.numel() < n or d_chars.numel() < h_chars.numel():
        raise ValueError("device buffers must be at least as large as the host arrays")
    for t in (h_out_perm, h_out_lcp):
        if t is not None and (t.is_cuda or t.dtype != torch.int32 or t.numel() < n or not t.is_contiguous()):
            raise ValueError("host outputs must be contiguous CPU int32 tensors of length >= n")
    ctx = ctx or context(d_chars.device.index)
    op, ol = _out(out_perm, n, d_chars.device), _out(out_lcp, n, d_chars.device)
    prm = prm or params()
    ctx._check(lib().sss_sort_host(ctx.h, _ptr(h_chars), h_chars.numel(), _ptr(h_offs), _ptr(h_lens), n, p,
                                   C.byref(prm), _ptr(d_chars), _ptr(d_offs), _ptr(d_lens), _ptr(op), _ptr(ol),
                                   _ptr(h_out_perm), _ptr(h_out_lcp)), ctx.h)
    return op, ol


NOALLOC_MAX_STRINGS = 65536


def sss_dist_prefix_noalloc(chars, offs, lens, prm: sss_params | None = None, out_approx=None):
    """Allocation-free stage B for at most NOALLOC_MAX_STRINGS strings, on the
    current torch stream (for callers that cannot allocate device memory; the
    output tensor must then be supplied by the caller)."""
    _check_strings(chars, offs, lens)
    n = lens.numel()
    if n > NOALLOC_MAX_STRINGS:  # checked here too: a count >= 2^32 would wrap in the C call
        raise ValueError(f"sss_dist_prefix_noalloc takes at most {NOALLOC_MAX_STRINGS} strings, got {n}")
    a = _out(out_approx, n, chars.device)
    prm = prm or params()
    # the C entry point works on the current CUDA device: make it the tensors' device
    with torch.cuda.device(chars.device):
        st = torch.cuda.current_stream(chars.device).cuda_stream
        status = lib().sss_dist_prefix_noalloc(_ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), n,
                                               C.byref(prm), _ptr(a), C.c_void_p(st))
    if status != 0:
        raise SssError(status, "sss_dist_prefix_noalloc failed")
    return a


def instance_table(first, sizes):
    """The sss_instance array (host) of instances (first[k], sizes[k], p = 1)."""
    import numpy as np
    m = len(first)
    rec = np.zeros(max(1, m), dtype=np.dtype([("first", "<u8"), ("n", "<u4"), ("p", "<u4")]))
    rec["first"][:m] = np.asarray(first, dtype=np.uint64)
    rec["n"][:m] = np.asarray(sizes, dtype=np.int64).astype(np.uint32)
    rec["p"][:m] = 1
    arr = (sss_instance * max(1, m)).from_buffer(rec)
    arr._keep = rec
    return arr, m


def sss_sort_batch(chars, offs, lens, first, sizes, prm: sss_params | None = None, out_perm=None, out_lcp=None,
                   want_dist: bool = False, ctx: Context | None = None):
    """Sort independent instances (strings first[k] .. first[k]+sizes[k]-1) of one
    string table together; returns (perm, lcp, dist or None), perm instance-local."""
    _check_strings(chars, offs, lens)
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    arr, m = instance_table(first, sizes)
    op, ol = _out(out_perm, n, chars.device), _out(out_lcp, n, chars.device)
    d = _out(None, n, chars.device) if want_dist else None
    prm = prm or params()
    ctx._check(lib().sss_sort_batch(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), n, arr, m,
                                    C.byref(prm), _ptr(op), _ptr(ol), _ptr(d)), ctx.h)
    return op, ol, d


def workspace_bytes(n: int, total_len: int, p: int = 1, prm: sss_params | None = None) -> int:
    prm = prm or params()
    return int(lib().sss_workspace_bytes(n, total_len, p, C.byref(prm)))


def sss_suffix_sort(text, max_len: int = 0, prm: sss_params | None = None, out_sa=None, out_lcp=None,
                    ctx: Context | None = None):
    """Suffix array and LCP array of a device uint8 text (suffix views, stage A)."""
    if not text.is_cuda or text.dtype != torch.uint8 or not text.is_contiguous():
        raise ValueError("text must be a contiguous CUDA uint8 tensor")
    ctx = ctx or context(text.device.index)
    n = text.numel()
    sa, lcp = _out(out_sa, n, text.device), _out(out_lcp, n, text.device)
    prm = prm or params()
    ctx._check(lib().sss_suffix_sort(ctx.h, _ptr(text), n, max_len, C.byref(prm), _ptr(sa), _ptr(lcp)), ctx.h)
    return sa, lcp


def batch_workspace_bytes(n_table: int, m: int, prm: sss_params | None = None) -> int:
    prm = prm or params()
    return int(lib().sss_batch_workspace_bytes(n_table, m, C.byref(prm)))


def to_device(ss, device="cuda"):
    """Copy a datagen.StringSet (numpy) to CUDA tensors (chars, offs, lens)."""
    import numpy as np
    chars = torch.from_numpy(ss.chars if ss.chars.size else np.zeros(1, np.uint8)).to(device)
    offs = torch.from_numpy(ss.offs.view(np.int64)).to(device)
    lens = torch.from_numpy(ss.lens.view(np.int32)).to(device)
    return chars, offs, lens


def u32(t: torch.Tensor):
    """A CUDA int32 tensor holding uint32 values, as a numpy uint32 array."""
    return t.cpu().numpy().view("uint32")
