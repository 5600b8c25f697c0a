"""CPU oracle for the string sorter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's product path never calls it
and shares no code with it (the C sources here are compiled on their own with
gcc into ``oracle/liboracle.so``).

Parity status: every function is pinned by ``tests/test_oracle_*.py``, the
64-bit prefix-hash values of ``prefix_key`` included (the paper fixes no hash
function; the one defined here is checked through the inverse of its finaliser
against the Karp-Rabin polynomial, its closed forms and its linearity).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_PAR = os.path.join(_HERE, "oracle_par.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
UINT32_MAX = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile oracle.c and oracle_par.c into liboracle.so with gcc (plain C, -O2)."""
    stale = (not os.path.exists(_SO) or
             os.path.getmtime(_SO) < max(os.path.getmtime(f) for f in (_SRC, _SRC_PAR, _HDR)))
    if force or stale:
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
        os.close(fd)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_PAR])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P8, P64, P32 = C.c_void_p, C.c_void_p, C.c_void_p
        u32, u64 = C.c_uint32, C.c_uint64
        sig = {
            "oracle_cmp": (C.c_int, [P8, P64, P32, P32, u32, u32]),
            "oracle_cmp_str": (C.c_int, [P8, P64, P32, P32, u32, u32]),
            "oracle_lcp_pair": (u32, [P8, P64, P32, P32, u32, u32]),
            "oracle_sort_idx": (None, [P8, P64, P32, P32, P32, u32]),
            "oracle_sort": (None, [P8, P64, P32, u32, P32]),
            "oracle_lcp_array": (None, [P8, P64, P32, P32, P32, u32, P32]),
            "oracle_dist": (None, [P32, u32, P32, P32, P32]),
            "oracle_mulmod61": (u64, [u64, u64]),
            "oracle_splitmix64_first": (u64, [u64]),
            "oracle_hash_base": (u64, [u64]),
            "oracle_prefix_key": (u64, [P8, P64, P32, u32, u32, u64]),
            "oracle_doubling": (None, [P8, P64, P32, u32, u32, u32, u64, P32, P32]),
            "oracle_part_lo": (u32, [u32, u32, u32]),
            "oracle_local_sort": (None, [P8, P64, P32, P32, u32, u32, P32, P32]),
            "oracle_samples": (u32, [P32, u32, u32, u32, P32]),
            "oracle_samples_char": (u32, [P32, P32, P32, u32, u32, u32, P32]),
            "oracle_splitters": (None, [P8, P64, P32, P32, P32, u32, u32, P32]),
            "oracle_bounds": (None, [P8, P64, P32, P32, P32, u32, u32, P32, P32]),
            "oracle_merge": (None, [P8, P64, P32, P32, P32, u32, u32, P32, P32, P32]),
            "oracle_check_sorted": (u32, [P8, P64, P32, P32, P32, u32]),
            "oracle_bounds_row": (None, [P8, P64, P32, P32, P32, u32, u32, P32, u32, P32]),
            "oracle_merge_bucket": (u32, [P8, P64, P32, P32, P32, u32, u32, P32, u32, P32]),
            "oracle_pdms_parallel": (C.c_int, [P8, P64, P32, u32, u32, u32, u32, u32, u64, u32, P32, P32, P32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _views(ss):
    chars = ss.chars if ss.chars.size else np.zeros(1, np.uint8)
    return chars, ss.offs, ss.lens


def sort(ss) -> np.ndarray:
    """perm[r] = input index of the r-th smallest string (ties by index)."""
    c, o, l = _views(ss)
    perm = np.empty(ss.n, np.uint32)
    lib().oracle_sort(_p(c), _p(o), _p(l), ss.n, _p(perm))
    return perm


def sort_idx(ss, idx, trunc=None) -> np.ndarray:
    c, o, l = _views(ss)
    idx = _u32(idx).copy()
    t = None if trunc is None else _u32(trunc)
    lib().oracle_sort_idx(_p(c), _p(o), _p(l), _p(t), _p(idx), idx.size)
    return idx


def lcp_array(ss, perm, trunc=None) -> np.ndarray:
    c, o, l = _views(ss)
    perm = _u32(perm)
    t = None if trunc is None else _u32(trunc)
    out = np.empty(perm.size, np.uint32)
    lib().oracle_lcp_array(_p(c), _p(o), _p(l), _p(t), _p(perm), perm.size, _p(out))
    return out


def lcp_pair(ss, a, b, trunc=None) -> int:
    c, o, l = _views(ss)
    t = None if trunc is None else _u32(trunc)
    return int(lib().oracle_lcp_pair(_p(c), _p(o), _p(l), _p(t), a, b))


def cmp(ss, a, b, trunc=None) -> int:
    c, o, l = _views(ss)
    t = None if trunc is None else _u32(trunc)
    return int(lib().oracle_cmp(_p(c), _p(o), _p(l), _p(t), a, b))


def dist(ss, perm, lcp) -> np.ndarray:
    out = np.empty(ss.n, np.uint32)
    lib().oracle_dist(_p(ss.lens), ss.n, _p(_u32(perm)), _p(_u32(lcp)), _p(out))
    return out


def mulmod61(a: int, b: int) -> int:
    return int(lib().oracle_mulmod61(a, b))


def splitmix64_first(s: int) -> int:
    return int(lib().oracle_splitmix64_first(s))


def hash_base(seed: int) -> int:
    return int(lib().oracle_hash_base(seed))


def prefix_key(ss, i: int, l: int, seed: int) -> int:
    c, o, ln = _views(ss)
    return int(lib().oracle_prefix_key(_p(c), _p(o), _p(ln), i, l, seed))


def doubling(ss, kmin: int, kmax: int, seed: int, want_rounds: bool = False):
    c, o, l = _views(ss)
    approx = np.empty(ss.n, np.uint32)
    rounds = np.zeros(kmax + 1, np.uint32)
    lib().oracle_doubling(_p(c), _p(o), _p(l), ss.n, kmin, kmax, seed, _p(approx), _p(rounds))
    return (approx, rounds) if want_rounds else approx


def part_lo(n: int, p: int, i: int) -> int:
    return (i * n) // p


def local_sort(ss, p: int, trunc=None):
    c, o, l = _views(ss)
    t = None if trunc is None else _u32(trunc)
    rp = np.empty(ss.n, np.uint32)
    rl = np.empty(ss.n, np.uint32)
    lib().oracle_local_sort(_p(c), _p(o), _p(l), _p(t), ss.n, p, _p(rp), _p(rl))
    return rp, rl


def samples(run_perm, n: int, p: int, v: int) -> np.ndarray:
    out = np.empty(p * (v + 1), np.uint32)
    ns = lib().oracle_samples(_p(_u32(run_perm)), n, p, v, _p(out))
    return out[:ns].copy()


def samples_char(ss, run_perm, p: int, v: int, trunc=None) -> np.ndarray:
    """Character-based regular sampling (Section 3.1.2)."""
    out = np.empty(p * (v + 1), np.uint32)
    t = None if trunc is None else _u32(trunc)
    ns = lib().oracle_samples_char(_p(_u32(ss.lens)), _p(t), _p(_u32(run_perm)), ss.n, p, v, _p(out))
    return out[:ns].copy()


def splitters(ss, smp, p: int, trunc=None):
    """Returns (sorted samples, splitters u32[p-1], UINT32_MAX = minus infinity)."""
    c, o, l = _views(ss)
    t = None if trunc is None else _u32(trunc)
    s = _u32(smp).copy()
    out = np.empty(max(p - 1, 1), np.uint32)
    lib().oracle_splitters(_p(c), _p(o), _p(l), _p(t), _p(s), s.size, p, _p(out))
    return s, out[:p - 1].copy()


def bounds(ss, run_perm, p: int, spl, trunc=None) -> np.ndarray:
    c, o, l = _views(ss)
    t = None if trunc is None else _u32(trunc)
    out = np.empty((p, p + 1), np.uint32)
    sp = _u32(spl) if p > 1 else np.zeros(1, np.uint32)
    lib().oracle_bounds(_p(c), _p(o), _p(l), _p(t), _p(_u32(run_perm)), ss.n, p, _p(sp), _p(out))
    return out


def merge(ss, run_perm, p: int, bnd, trunc=None):
    c, o, l = _views(ss)
    t = None if trunc is None else _u32(trunc)
    op = np.empty(ss.n, np.uint32)
    ol = np.empty(ss.n, np.uint32)
    lib().oracle_merge(_p(c), _p(o), _p(l), _p(t), _p(_u32(run_perm)), ss.n, p,
                       _p(_u32(bnd)), _p(op), _p(ol))
    return op, ol


def check_sorted(ss, perm, lcp) -> int:
    c, o, l = _views(ss)
    return int(lib().oracle_check_sorted(_p(c), _p(o), _p(l), _p(_u32(perm)), _p(_u32(lcp)), ss.n))


def pdms(ss, p: int, v: int = 2, kmin: int = 0, kmax: int | None = None, seed: int = 0,
         char_sampling: bool = False):
    """The prefix-doubling merge sort pipeline step by step (Sections 3 and 4):
    local sort of each partition, prefix doubling, regular sampling (string-based,
    or character-based on the approx-truncated lengths, Section 3.1.2),
    splitters, bucket bounds, and the merge of the buckets on approx-truncated
    strings.  Returns a dict with every intermediate array."""
    if kmax is None:
        kmax = default_kmax(ss)
    run_perm, run_lcp = local_sort(ss, p)
    approx = doubling(ss, kmin, kmax, seed)
    smp = samples_char(ss, run_perm, p, v, approx) if char_sampling else samples(run_perm, ss.n, p, v)
    sorted_smp, spl = splitters(ss, smp, p, approx)
    bnd = bounds(ss, run_perm, p, spl, approx)
    perm, lcp = merge(ss, run_perm, p, bnd, approx)
    return dict(run_perm=run_perm, run_lcp=run_lcp, approx=approx, samples=smp,
                sorted_samples=sorted_smp, splitters=spl, bounds=bnd, perm=perm, lcp=lcp)


def pdms_parallel(ss, p: int, v: int = 2, kmin: int = 0, kmax: int | None = None, seed: int = 0,
                  nthreads: int | None = None):
    """The same pipeline as pdms() (string-based sampling) on nthreads host
    threads (default: every core); returns (perm, lcp, approx), equal to pdms()'s."""
    if kmax is None:
        kmax = default_kmax(ss)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    c, o, l = _views(ss)
    perm = np.empty(ss.n, np.uint32)
    lcp = np.empty(ss.n, np.uint32)
    approx = np.empty(ss.n, np.uint32)
    rc = lib().oracle_pdms_parallel(_p(c), _p(o), _p(l), ss.n, p, v, kmin, kmax, seed, nthreads, _p(perm), _p(lcp),
                                    _p(approx))
    if rc != 0:
        raise RuntimeError("oracle_pdms_parallel: a thread could not be started")
    return perm, lcp, approx


def default_kmax(ss) -> int:
    """kmax = ceil(log2(max length)) (0 for sets of empty or 1-char strings)."""
    m = int(ss.lens.max()) if ss.n else 0
    k = 0
    while (1 << k) < m:
        k += 1
    return k
