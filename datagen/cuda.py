"""Device-side generation of the template string sets of ``datagen`` (same
definitions, produced directly in CUDA memory).  Built with nvcc into
``datagen/libsssgen.so``; used by the benchmark for full-size workloads and
checked against the numpy generator by the GPU tests."""
from __future__ import annotations

import ctypes as C
import threading
import os
import subprocess
import tempfile

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_cuda.cu")
_SO = os.path.join(_HERE, "libsssgen.so")


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        from paper_2404_16517_gb300 import _build as b
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
        os.close(fd)
        cmd = [b.nvcc(), *b.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
               "-o", tmp, _SRC, "-Xlinker", f"-rpath,{b.cuda_lib_dir()}", "-L", b.cuda_lib_dir()]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


_lib = None


_lib_lock = threading.Lock()


def lib():
    """The generator library, loaded once; the handle is published only after
    every signature is set (several threads may ask for it at once)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is None:
            _lib = _configure(C.CDLL(build()))
    return _lib


def _configure(_lib):
    g = _lib.sssgen_instance_chars
    g.restype = C.c_int
    g.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64,
                  C.c_char_p, C.c_uint32, C.c_void_p]
    h = _lib.sssgen_request
    h.restype = C.c_int
    h.argtypes = [C.c_void_p] * 5 + [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double, C.c_uint32,
                                     C.c_char_p, C.c_uint32, C.c_uint64, C.c_void_p]
    _lib.sssgen_request_scratch_words.restype = C.c_uint64
    _lib.sssgen_request_totals.restype = C.c_int
    _lib.sssgen_request_totals.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint32,
                                           C.c_void_p, C.c_void_p]
    _lib.sssgen_request_scratch_words.argtypes = [C.c_uint64]
    _lib.sssgen_skew_chars.restype = C.c_int
    _lib.sssgen_skew_chars.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint32,
                                       C.c_char_p, C.c_uint32, C.c_void_p]
    _lib.sssgen_req_desc_bytes.restype = C.c_uint32
    _lib.sssgen_req_desc_bytes.argtypes = []
    _lib.sssgen_request_batch.restype = C.c_int
    _lib.sssgen_request_batch.argtypes = [C.c_void_p] * 6 + [C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32,
                                                              C.c_char_p, C.c_uint32, C.c_void_p]
    f = _lib.sssgen_template_set
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                  C.c_uint32, C.c_char_p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_void_p]
    return _lib


def template_set(seed: int, n: int, length: int, n_templates: int, shared: int, alphabet: bytes,
                 first: int = 0, count: int | None = None, device: str = "cuda"):
    """Device tensors (chars u8, offs i64, lens i32) of strings first..first+count-1."""
    import torch
    if count is None:
        count = n - first
    chars = torch.empty(max(1, count * length), dtype=torch.uint8, device=device)
    offs = torch.empty(count, dtype=torch.int64, device=device)
    lens = torch.empty(count, dtype=torch.int32, device=device)
    st = torch.cuda.current_stream(chars.device).cuda_stream
    rc = lib().sssgen_template_set(C.c_void_p(chars.data_ptr()), C.c_void_p(offs.data_ptr()),
                                   C.c_void_p(lens.data_ptr()), seed, n, length, n_templates, shared, alphabet,
                                   len(alphabet), first, count, C.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"sssgen_template_set failed ({rc})")
    return chars, offs, lens


def config2(n: int = 4194304, first: int = 0, count: int | None = None, device: str = "cuda"):
    return template_set(2, n, 500, 64, 242, b"ABCDEFGHIJKLMNOPQRSTUVWXYZ", first, count, device)


def config1(device: str = "cuda"):
    return template_set(1, 65536, 100, 4, 42, b"ABCDEFGHIJKLMNOPQRSTUVWXYZ", 0, None, device)


def instance_set(seed: int, sizes, len_lo: int, len_hi: int, ratios, alphabet: bytes = b"ACGT", device: str = "cuda"):
    """Device tensors (chars, offs, lens) and first (numpy u64[m+1]) of an
    instance set, byte-identical to datagen.instance_set."""
    import numpy as np
    import torch

    import datagen
    first, lens, offs, cp, inst = datagen.instance_layout(seed, np.asarray(sizes), len_lo, len_hi,
                                                           np.asarray(ratios, dtype=np.float64), len(alphabet))
    n = lens.shape[0]
    N = int(lens.astype(np.uint64).sum())
    chars = torch.empty(max(1, N), dtype=torch.uint8, device=device)
    t_offs = torch.from_numpy(offs.view(np.int64)).to(device)
    t_lens = torch.from_numpy(lens.view(np.int32)).to(device)
    t_cp = torch.from_numpy(cp.view(np.int32)).to(device)
    t_inst = torch.from_numpy(inst.view(np.int32)).to(device)
    st = torch.cuda.current_stream(chars.device).cuda_stream
    rc = lib().sssgen_instance_chars(C.c_void_p(chars.data_ptr()), C.c_void_p(t_offs.data_ptr()),
                                     C.c_void_p(t_lens.data_ptr()), C.c_void_p(t_cp.data_ptr()),
                                     C.c_void_p(t_inst.data_ptr()), n, seed, alphabet, len(alphabet), C.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"sssgen_instance_chars failed ({rc})")
    return chars, t_offs, t_lens, first


def config4(m: int = 4096, size_cap: int | None = None, device: str = "cuda"):
    import numpy as np

    import datagen
    sizes, r = datagen.config4_sizes(4, m)
    if size_cap is not None:
        sizes = np.minimum(sizes, size_cap)
    return instance_set(4, sizes, 8, 300, r, b"ACGT", device)


def request_scratch_words(n: int) -> int:
    """uint64 words of sum scratch that request_into needs for n strings."""
    return int(lib().sssgen_request_scratch_words(n))


def request_into(chars, char_base: int, offs, lens, cp_scratch, sum_scratch, seed: int, n: int, ratio: float,
                 len_lo: int = 16, len_hi: int = 1000, alphabet: bytes = b"ABCDEFGHIJKLMNOPQRSTUVWXYZ"):
    """Generate one serving request (n strings, lengths uniform len_lo..len_hi,
    template copy ratio `ratio`) on the device, on the current stream, without a
    host synchronisation: lens[0:n], offs[0:n] (absolute, starting at
    char_base) and chars[char_base : char_base + request_chars(seed, n)].
    cp_scratch: >= n int32; sum_scratch: >= request_scratch_words(n) int64.
    The characters depend on (seed, n, ratio) only, not on char_base."""
    import math

    import torch
    if n == 0:
        return
    assert cp_scratch.numel() >= n and sum_scratch.numel() >= request_scratch_words(n)
    assert offs.numel() >= n and lens.numel() >= n
    st = torch.cuda.current_stream(lens.device).cuda_stream
    logs = int(math.ceil(math.log(max(n, 2)) / math.log(len(alphabet))))
    rc = lib().sssgen_request(C.c_void_p(chars.data_ptr()), C.c_void_p(offs.data_ptr()),
                              C.c_void_p(lens.data_ptr()), C.c_void_p(cp_scratch.data_ptr()),
                              C.c_void_p(sum_scratch.data_ptr()), n, seed & ((1 << 64) - 1), len_lo, len_hi,
                              float(ratio), logs, alphabet, len(alphabet), char_base, C.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"sssgen_request failed ({rc})")


def request_totals(seeds, sizes, len_lo: int = 16, len_hi: int = 1000, device: str = "cuda"):
    """Total characters of each serving request (numpy int64[m]), computed on
    the device with the generator's own length draws."""
    import numpy as np
    import torch
    m = len(seeds)
    if m == 0:
        return np.zeros(0, dtype=np.int64)
    t_seeds = torch.from_numpy(np.asarray(seeds, dtype=np.uint64).view(np.int64)).to(device)
    t_ns = torch.from_numpy(np.asarray(sizes, dtype=np.int64)).to(device)
    out = torch.empty(m, dtype=torch.int64, device=device)
    st = torch.cuda.current_stream(out.device).cuda_stream
    rc = lib().sssgen_request_totals(C.c_void_p(t_seeds.data_ptr()), C.c_void_p(t_ns.data_ptr()), m, len_lo, len_hi,
                                     C.c_void_p(out.data_ptr()), C.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"sssgen_request_totals failed ({rc})")
    return out.cpu().numpy()


def _req_desc_dtype():
    import numpy as np
    return np.dtype([("kl", "<u8"), ("kt", "<u8"), ("kc", "<u8"), ("char_base", "<u8"), ("ratio", "<f8"),
                     ("first", "<u4"), ("n", "<u4"), ("logs", "<u4"), ("pad", "<u4")])


def request_descs(seeds, sizes, ratios, char_bases, alphabet_len: int = 26):
    """Host descriptor table (numpy) of a batch of requests packed back to back
    into one string table, for request_batch_into."""
    import math

    import numpy as np

    import datagen
    dt = _req_desc_dtype()
    assert dt.itemsize == int(lib().sssgen_req_desc_bytes())
    m = len(seeds)
    d = np.zeros(m, dtype=dt)
    f = 0
    for k in range(m):
        sd, n = int(seeds[k]) & ((1 << 64) - 1), int(sizes[k])
        d[k] = (datagen.stream_key(sd, datagen.ST_LEN), datagen.stream_key(sd, datagen.ST_TEMPLATE),
                datagen.stream_key(sd, datagen.ST_CHARS), int(char_bases[k]), float(ratios[k]), f, n,
                int(math.ceil(math.log(max(n, 2)) / math.log(alphabet_len))), 0)
        f += n
    return d


def request_batch_into(chars, offs, lens, cp_scratch, sum_scratch, desc_dev, m: int, n: int, len_lo: int = 16,
                       len_hi: int = 1000, alphabet: bytes = b"ABCDEFGHIJKLMNOPQRSTUVWXYZ"):
    """Generate every request of a batch (descriptors already on the device,
    desc_dev) into one table in a single launch sequence on the current stream;
    request k gets the strings request_into would give it.  cp_scratch: >= n
    int32; sum_scratch: >= request_scratch_words(n) + m int64."""
    import torch
    if n == 0:
        return
    assert cp_scratch.numel() >= n and sum_scratch.numel() >= request_scratch_words(n) + m
    st = torch.cuda.current_stream(lens.device).cuda_stream
    rc = lib().sssgen_request_batch(C.c_void_p(chars.data_ptr()), C.c_void_p(offs.data_ptr()),
                                    C.c_void_p(lens.data_ptr()), C.c_void_p(cp_scratch.data_ptr()),
                                    C.c_void_p(sum_scratch.data_ptr()), C.c_void_p(desc_dev.data_ptr()), m, n, len_lo,
                                    len_hi, alphabet, len(alphabet), C.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"sssgen_request_batch failed ({rc})")


def skew_set(seed: int = 6, n: int = 1 << 22, short: int = 20, long: int = 1000, device: str = "cuda"):
    """Device tensors (chars, offs, lens) of datagen.skew_set, byte-identical."""
    import numpy as np
    import torch

    import datagen
    alphabet = b"ABCDEFGHIJKLMNOPQRSTUVWXYZ"
    _, lens, offs = datagen.skew_layout(seed, n, short, long, len(alphabet))
    N = int(lens.astype(np.uint64).sum())
    chars = torch.empty(max(1, N), dtype=torch.uint8, device=device)
    t_offs = torch.from_numpy(offs.view(np.int64)).to(device)
    t_lens = torch.from_numpy(lens.view(np.int32)).to(device)
    st = torch.cuda.current_stream(chars.device).cuda_stream
    rc = lib().sssgen_skew_chars(C.c_void_p(chars.data_ptr()), C.c_void_p(t_offs.data_ptr()),
                                 C.c_void_p(t_lens.data_ptr()), n, seed, long, alphabet, len(alphabet),
                                 C.c_void_p(st))
    if rc != 0:
        raise RuntimeError(f"sssgen_skew_chars failed ({rc})")
    return chars, t_offs, t_lens
