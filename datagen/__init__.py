"""Seeded synthetic string sets for the string sorter and its oracle.

This module holds the input generators only: it contains none of the sorting
method's arithmetic (no comparisons, no LCPs, no hashing of prefixes).  Both the
CPU oracle tests and the CUDA path draw their inputs from here, so the two sides
always see byte-identical data.

Randomness is counter-based: ``rng(seed, stream, i)`` is the i-th output of a
SplitMix64 sequence (Steele, Lea, Flood 2014) whose seed is itself the
``stream``-th output of the SplitMix64 sequence started at ``seed``:

    smix(z)     = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
                  z *= 0x94D049BB133111EB; z ^ (z>>31)          (mod 2^64)
    rng(s,t,i)  = smix(smix(s + (t+1)*G) + (i+1)*G),  G = 0x9E3779B97F4A7C15

A uniform draw from an alphabet of size A takes the high 32 bits of ``rng`` and
maps them with a multiply-shift, ``((r >> 32) * A) >> 32``.  The CUDA generator
in ``datagen/gen_cuda.cu`` implements the same definitions, so large sets can be
produced directly in device memory.

The string sets follow the shapes of the paper's DNData workload (Section 5,
"DNGenerator", length-500 strings with D/N near 0.5): every string copies a
prefix from one of a few seeded templates and continues with uniform random
characters, so the shared template prefix controls the distinguishing prefix.

A string set is the triple ``(chars u8[N], offs u64[n], lens u32[n])``: string i
is ``chars[offs[i] : offs[i] + lens[i]]``.  No string contains the byte 0x00.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1

# stream ids (arbitrary distinct constants)
ST_TEMPLATE = 1
ST_PICK = 2
ST_CHARS = 3
ST_LEN = 4
ST_MARKOV = 5
ST_OFFSET = 6
ST_SIZE = 7
ST_RATIO = 8

UPPER = np.frombuffer(b"ABCDEFGHIJKLMNOPQRSTUVWXYZ", dtype=np.uint8)
DNA = np.frombuffer(b"ACGT", dtype=np.uint8)

_U = np.uint64


def _smix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U(30))) * _U(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U(27))) * _U(0x94D049BB133111EB)
        return z ^ (z >> _U(31))


def smix_int(z: int) -> int:
    """Scalar SplitMix64 output function on a Python int (mod 2^64)."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return smix_int((seed + (stream + 1) * GAMMA) & M64)


def rng(seed: int, stream: int, i) -> np.ndarray:
    """Counter-based draw ``rng(seed, stream, i)`` for an array of counters ``i``."""
    k = _U(stream_key(seed, stream))
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _smix(k + (i + _U(1)) * _U(GAMMA))


def uniform_index(r: np.ndarray, a: int) -> np.ndarray:
    """Map 64-bit draws to [0, a) by multiply-shift on the high 32 bits."""
    with np.errstate(over="ignore"):
        return ((r >> _U(32)) * _U(a)) >> _U(32)


def uniform_float(r: np.ndarray) -> np.ndarray:
    """Map 64-bit draws to [0, 1) using the top 53 bits."""
    return (r >> _U(11)).astype(np.float64) * (1.0 / (1 << 53))


class StringSet:
    """A string set in (chars, offs, lens) form plus a few shape statistics."""

    def __init__(self, chars: np.ndarray, offs: np.ndarray, lens: np.ndarray, name: str = ""):
        self.chars = np.ascontiguousarray(chars, dtype=np.uint8)
        self.offs = np.ascontiguousarray(offs, dtype=np.uint64)
        self.lens = np.ascontiguousarray(lens, dtype=np.uint32)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.lens.shape[0])

    @property
    def N(self) -> int:
        """Total characters over all strings (overlapping views counted in full)."""
        return int(self.lens.astype(np.uint64).sum())

    def string(self, i: int) -> bytes:
        o = int(self.offs[i])
        return self.chars[o:o + int(self.lens[i])].tobytes()

    def strings(self) -> list[bytes]:
        return [self.string(i) for i in range(self.n)]


def from_strings(strs: list[bytes], name: str = "") -> StringSet:
    """Pack a Python list of byte strings (no 0x00 inside) into a StringSet."""
    lens = np.array([len(s) for s in strs], dtype=np.uint32)
    offs = np.zeros(len(strs), dtype=np.uint64)
    if len(strs) > 1:
        offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    chars = np.frombuffer(b"".join(strs), dtype=np.uint8).copy() if strs else np.zeros(0, np.uint8)
    for s in strs:
        assert b"\x00" not in s
    return StringSet(chars, offs, lens, name)


def template_set(seed: int, n: int, length: int, n_templates: int, shared: int,
                 alphabet: np.ndarray = UPPER, first: int = 0, count: int | None = None) -> StringSet:
    """Fixed-length strings: ``shared`` chars from one of ``n_templates`` seeded
    templates (picked uniformly per string), the rest uniform random.

    Strings ``first .. first+count-1`` of the full n-string set are produced (so a
    bounded sample of a large set is byte-identical to the same strings of the
    full set); offsets are relative to the returned chars array.
    """
    if count is None:
        count = n - first
    a = int(alphabet.shape[0])
    tmpl = alphabet[uniform_index(rng(seed, ST_TEMPLATE, np.arange(n_templates * length, dtype=np.uint64)), a)]
    tmpl = tmpl.reshape(n_templates, length)
    ids = np.arange(first, first + count, dtype=np.uint64)
    pick = uniform_index(rng(seed, ST_PICK, ids), n_templates).astype(np.int64)
    chars = np.empty((count, length), dtype=np.uint8)
    # uniform part: counter = i*length + j
    step = max(1, (1 << 22) // max(1, length))
    for b in range(0, count, step):
        e = min(count, b + step)
        cnt = (ids[b:e, None] * _U(length) + np.arange(length, dtype=np.uint64)[None, :])
        chars[b:e] = alphabet[uniform_index(rng(seed, ST_CHARS, cnt), a)]
    if shared > 0:
        chars[:, :shared] = tmpl[pick, :shared]
    offs = np.arange(count, dtype=np.uint64) * _U(length)
    lens = np.full(count, length, dtype=np.uint32)
    return StringSet(chars.reshape(-1), offs, lens, f"template(seed={seed},n={n},len={length},T={n_templates},shared={shared})")


def config1(first: int = 0, count: int | None = None) -> StringSet:
    """Plain-sort workload: 65,536 strings of 100 chars over A-Z; chars 0-41 from
    one of 4 templates, the rest uniform (D/N near 0.5)."""
    return template_set(1, 65536, 100, 4, 42, UPPER, first, count)


def config2(n: int = 4194304, first: int = 0, count: int | None = None) -> StringSet:
    """Full-pipeline workload: 4,194,304 strings of 500 chars over A-Z; chars
    0-241 from one of 64 templates, the rest uniform (D/N near 0.5).  ``n`` may be
    reduced for scaled-down cases."""
    return template_set(2, n, 500, 64, 242, UPPER, first, count)


def markov_text(seed: int, length: int, sigma: int = 64, alpha: float = 0.1) -> np.ndarray:
    """Order-2 Markov text over ``sigma`` symbols (bytes 0x21 + symbol).

    Transition rows are Dirichlet(alpha) draws from numpy's PCG64 seeded with
    ``seed`` (the one place this module uses numpy's generator); each step draws
    one counter-based uniform and inverts the row's CDF.
    """
    g = np.random.Generator(np.random.PCG64(seed))
    rows = g.dirichlet(np.full(sigma, alpha), size=sigma * sigma)
    cdf = np.cumsum(rows, axis=1)
    cdf[:, -1] = 1.0
    u = uniform_float(rng(seed, ST_MARKOV, np.arange(length, dtype=np.uint64)))
    first2 = uniform_index(rng(seed, ST_MARKOV, np.arange(length, length + 2, dtype=np.uint64)), sigma)
    import bisect
    rows = cdf.tolist()
    uu = u.tolist()
    sym = [0] * length
    sym[0] = int(first2[0])
    if length > 1:
        sym[1] = int(first2[1])
    # sequential chain: invert the row's CDF at one uniform per step
    a, b = sym[0], sym[1] if length > 1 else 0
    last = sigma - 1
    for t in range(2, length):
        c = bisect.bisect_right(rows[a * sigma + b], uu[t])
        if c > last:
            c = last
        sym[t] = c
        a, b = b, c
    sym = np.asarray(sym, dtype=np.int64)
    return (sym + 0x21).astype(np.uint8)


def suffix_set(seed: int = 3, text_len: int = 1 << 22, n: int = 1 << 21, max_len: int = 256,
               text: np.ndarray | None = None) -> StringSet:
    """Suffix-like high-LCP set: ``n`` distinct random offsets into a Markov text,
    each suffix truncated to ``max_len`` chars (strings are views into one text)."""
    if text is None:
        text = markov_text(seed, text_len)
    keys = rng(seed, ST_OFFSET, np.arange(text_len, dtype=np.uint64))
    order = np.argsort(keys, kind="stable")
    offs = np.sort(order[:n]).astype(np.uint64)
    # keep a seeded order that is not sorted by offset
    perm = np.argsort(rng(seed, ST_OFFSET + 100, np.arange(n, dtype=np.uint64)), kind="stable")
    offs = offs[perm]
    lens = np.minimum(np.uint64(max_len), np.uint64(text_len) - offs).astype(np.uint32)
    return StringSet(text, offs, lens, f"suffix(seed={seed},text={text_len},n={n},max={max_len})")


def config3(scale: int = 0) -> StringSet:
    """Suffix workload: text of 2^22 bytes, 2^21 suffixes, length <= 256.
    ``scale`` > 0 divides both sizes by 2^scale for scaled-down cases."""
    return suffix_set(3, (1 << 22) >> scale, (1 << 21) >> scale, 256)


def instance_layout(seed: int, sizes: np.ndarray, len_lo: int, len_hi: int, ratios: np.ndarray, a: int):
    """Per-string layout of an instance set: (first u64[m+1], lens, offs, copy
    lengths, instance ids).  String g of instance k copies
    max(0, round(r_k*len) - ceil(log_a n_k) - 1) template characters."""
    sizes = np.asarray(sizes, dtype=np.int64)
    m = sizes.shape[0]
    first = np.zeros(m + 1, dtype=np.uint64)
    first[1:] = np.cumsum(sizes).astype(np.uint64)
    n = int(first[-1])
    gid = np.arange(n, dtype=np.uint64)
    inst = np.repeat(np.arange(m, dtype=np.int64), sizes)
    lens = (len_lo + uniform_index(rng(seed, ST_LEN, gid), len_hi - len_lo + 1)).astype(np.uint32)
    logs = np.ceil(np.log(np.maximum(sizes, 2)) / np.log(a)).astype(np.int64)
    cp = np.maximum(0, np.rint(ratios[inst] * lens).astype(np.int64) - logs[inst] - 1)
    cp = np.minimum(cp, lens.astype(np.int64))
    offs = np.zeros(n, dtype=np.uint64)
    if n > 1:
        offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    return first, lens, offs, cp.astype(np.uint32), inst.astype(np.uint32)


def instance_set(seed: int, sizes: np.ndarray, len_lo: int, len_hi: int, ratios: np.ndarray,
                 alphabet: np.ndarray = DNA) -> tuple[StringSet, np.ndarray]:
    """Independent sort instances packed into one string table.

    Instance k has ``sizes[k]`` strings with lengths uniform in [len_lo, len_hi];
    string j of instance k copies ``max(0, round(r_k*len) - ceil(log_A n_k) - 1)``
    chars of the instance's template, then continues uniformly.  Returns the set and
    ``first`` (u64[m+1]): instance k is strings ``first[k] .. first[k+1]-1``.
    """
    a = int(alphabet.shape[0])
    first, lens, offs, cp, inst = instance_layout(seed, sizes, len_lo, len_hi, ratios, a)
    n = lens.shape[0]
    N = int(lens.astype(np.uint64).sum())
    pos_in = np.arange(N, dtype=np.int64) - np.repeat(offs.astype(np.int64), lens.astype(np.int64))
    owner = np.repeat(np.arange(n, dtype=np.int64), lens.astype(np.int64))
    rand = alphabet[uniform_index(rng(seed, ST_CHARS, np.arange(N, dtype=np.uint64)), a)]
    tmpl_cnt = inst[owner].astype(np.uint64) * _U(1 << 20) + pos_in.astype(np.uint64)
    tmpl = alphabet[uniform_index(rng(seed, ST_TEMPLATE, tmpl_cnt), a)]
    chars = np.where(pos_in < cp[owner].astype(np.int64), tmpl, rand).astype(np.uint8)
    ss = StringSet(chars, offs, lens, f"instances(seed={seed},m={sizes.shape[0]},n={n})")
    return ss, first


def config4_sizes(seed: int = 4, m: int = 4096) -> tuple[np.ndarray, np.ndarray]:
    """Batched workload shape: sizes log-uniform over 2^6..2^16, D/N ratio uniform
    over 0.1..0.9 per instance."""
    u = uniform_float(rng(seed, ST_SIZE, np.arange(m, dtype=np.uint64)))
    sizes = np.floor(2.0 ** (6.0 + 10.0 * u)).astype(np.int64)
    r = 0.1 + 0.8 * uniform_float(rng(seed, ST_RATIO, np.arange(m, dtype=np.uint64)))
    return sizes, r


def config4(m: int = 4096, size_cap: int | None = None) -> tuple[StringSet, np.ndarray]:
    """Batched workload: ``m`` instances, lengths uniform 8..300 over {A,C,G,T}."""
    sizes, r = config4_sizes(4, m)
    if size_cap is not None:
        sizes = np.minimum(sizes, size_cap)
    return instance_set(4, sizes, 8, 300, r, DNA)


def config5_requests(count: int = 20000, seed: int = 5, median_log2: float = 14.0, sigma: float = 1.5,
                     cap: int = 1 << 24):
    """Serving workload shape: request sizes lognormal (median 2^14 strings,
    sigma 1.5, capped at 2^24), copy ratio uniform over 0.1..0.9, and unit-rate
    exponential inter-arrival gaps (scale them by 1/lambda).  Normal draws use
    Box-Muller on counter-based uniforms.  Returns (sizes, ratios, gaps, seeds)."""
    i = np.arange(count, dtype=np.uint64)
    u1 = uniform_float(rng(seed, ST_SIZE, i))
    u2 = uniform_float(rng(seed, ST_SIZE + 100, i))
    z = np.sqrt(-2.0 * np.log(np.maximum(u1, 1e-300))) * np.cos(2.0 * np.pi * u2)
    sizes = np.minimum(cap, np.maximum(1, np.rint(2.0 ** median_log2 * np.exp(sigma * z)))).astype(np.int64)
    ratios = 0.1 + 0.8 * uniform_float(rng(seed, ST_RATIO, i))
    gaps = -np.log(np.maximum(1.0 - uniform_float(rng(seed, ST_OFFSET, i)), 1e-300))
    seeds = rng(seed, ST_TEMPLATE + 100, i)
    return sizes, ratios, gaps, seeds


def request_chars(seed: int, n: int, len_lo: int = 16, len_hi: int = 1000, chunk: int = 1 << 22) -> int:
    """Total characters of a serving request of n strings (the sum of the same
    length draws the device generator makes), computed on the host."""
    tot = 0
    for a in range(0, n, chunk):
        i = np.arange(a, min(n, a + chunk), dtype=np.uint64)
        tot += int((len_lo + uniform_index(rng(seed, ST_LEN, i), len_hi - len_lo + 1)).sum())
    return tot


def skew_layout(seed: int, n: int, short: int = 20, long: int = 1000, a: int = 26):
    """Length-skewed set layout: string i starts with letter uniform_index(rng(seed,
    ST_PICK, i), a); strings starting with the last letter have `long`
    characters, the others `short`.  Returns (first letter index, lens, offs)."""
    first = uniform_index(rng(seed, ST_PICK, np.arange(n, dtype=np.uint64)), a).astype(np.uint32)
    lens = np.where(first == a - 1, long, short).astype(np.uint32)
    offs = np.zeros(n, dtype=np.uint64)
    if n > 1:
        offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    return first, lens, offs


def skew_set(seed: int = 6, n: int = 1 << 22, short: int = 20, long: int = 1000,
             alphabet: np.ndarray = UPPER) -> StringSet:
    """Strings whose sort order and distinguishing-prefix length are correlated,
    the case character-based sampling is for: first letter as in skew_layout;
    a long string (last letter first) copies characters 1 .. long-9 from one
    seeded template and ends in 8 uniform characters, so all long strings share
    long-8 characters and sort last; short strings are uniform after their
    first letter (counter = offset + j; template counter = j)."""
    a = int(alphabet.shape[0])
    first, lens, offs = skew_layout(seed, n, short, long, a)
    N = int(lens.astype(np.uint64).sum())
    chars = alphabet[uniform_index(rng(seed, ST_CHARS, np.arange(N, dtype=np.uint64)), a)]
    tmpl = alphabet[uniform_index(rng(seed, ST_TEMPLATE, np.arange(long, dtype=np.uint64)), a)]
    for i in np.nonzero(first == a - 1)[0]:
        o = int(offs[i])
        chars[o + 1: o + long - 8] = tmpl[1: long - 8]
    chars[offs.astype(np.int64)] = alphabet[first]
    return StringSet(chars, offs, lens, f"skew(seed={seed},n={n})")
