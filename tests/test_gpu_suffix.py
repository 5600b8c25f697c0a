"""Suffix sorting through sss_suffix_sort (suffix views of one text sorted by
stage A, then prefix doubling over ranks where 64 characters do not separate
them): the suffix array and LCP array equal Python's sort of the suffixes on
small texts (repetitive ones included, so that several doubling rounds run, with
truncation lengths on and off the doubling lengths) and the oracle's sort of the
suffix views on a Markov text and on a long-period repetitive text, whole and
truncated; a text of one repeated character matches its closed form quickly."""
import random

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sss():
    import paper_2404_16517_gb300 as m
    return m


def py_sa(text: bytes, max_len: int = 0):
    n = len(text)
    key = (lambda i: text[i:i + max_len]) if max_len else (lambda i: text[i:])
    sa = sorted(range(n), key=lambda i: (key(i), i))
    lcp = [0] * n
    for r in range(1, n):
        a, b = key(sa[r - 1]), key(sa[r])
        k = 0
        while k < min(len(a), len(b)) and a[k] == b[k]:
            k += 1
        lcp[r] = k
    return np.array(sa, np.uint32), np.array(lcp, np.uint32)


def _planted(seed: int, n: int, unit: int) -> bytes:
    """Random ACGT text made of copies of a few random blocks (long repeats)."""
    rnd = random.Random(seed)
    blocks = [bytes(rnd.choice(b"ACGT") for _ in range(unit)) for _ in range(3)]
    out = b""
    while len(out) < n:
        out += rnd.choice(blocks) if rnd.random() < 0.8 else bytes(rnd.choice(b"ACGT") for _ in range(7))
    return out[:n]


CASES = [b"banana", b"A", b"AB", b"mississippi", b"A" * 1500, b"AB" * 900, b"ABC" * 400 + b"ABD",
         bytes(random.Random(1).choice(b"AC") for _ in range(3000)),
         bytes(random.Random(2).choice(b"ACGT") for _ in range(5000)),
         b"A" * 700 + b"B" + b"A" * 700, (b"ACGTACGTTG" * 200)[:1999] + b"C", _planted(3, 4000, 150)]


@pytest.mark.parametrize("i", range(len(CASES)))
@pytest.mark.parametrize("max_len", [0, 7, 64, 100, 200])
def test_suffix_array_small(i, max_len):
    m = sss()
    text = CASES[i]
    sa, lcp = m.sss_suffix_sort(torch.tensor(list(text), dtype=torch.uint8, device="cuda"), max_len)
    m.context().sync()
    want_sa, want_lcp = py_sa(text, max_len)
    assert np.array_equal(m.u32(sa), want_sa)
    assert np.array_equal(m.u32(lcp), want_lcp)


@pytest.mark.parametrize("max_len", [0, 256])
def test_suffix_array_markov_text(max_len):
    m = sss()
    text = datagen.markov_text(3, 1 << 17)
    n = text.shape[0]
    offs = np.arange(n, dtype=np.uint64)
    lens = (n - offs).astype(np.uint32)
    if max_len:
        lens = np.minimum(lens, max_len).astype(np.uint32)
    ss = datagen.StringSet(text, offs, lens)
    want = oracle.sort(ss)
    sa, lcp = m.sss_suffix_sort(torch.from_numpy(text).cuda(), max_len)
    m.context().sync()
    assert np.array_equal(m.u32(sa), want)
    assert np.array_equal(m.u32(lcp), oracle.lcp_array(ss, want))


def test_suffix_checked_rejects_nul():
    m = sss()
    t = torch.tensor(list(b"AB\x00CD"), dtype=torch.uint8, device="cuda")
    with pytest.raises(m.SssError):
        m.sss_suffix_sort(t, 0, m.params(flags=m.SSS_FLAG_CHECKED))
        m.context().sync()


def test_suffix_array_repetitive_text_vs_oracle():
    """A long-period repetitive text (several doubling rounds) against the oracle."""
    m = sss()
    text = np.frombuffer(_planted(7, 60000, 1000), dtype=np.uint8).copy()
    n = text.shape[0]
    for max_len in (0, 3000):
        offs = np.arange(n, dtype=np.uint64)
        lens = (n - offs).astype(np.uint32)
        if max_len:
            lens = np.minimum(lens, max_len).astype(np.uint32)
        ss = datagen.StringSet(text, offs, lens)
        want = oracle.sort(ss)
        sa, lcp = m.sss_suffix_sort(torch.from_numpy(text).cuda(), max_len)
        m.context().sync()
        assert np.array_equal(m.u32(sa), want)
        assert np.array_equal(m.u32(lcp), oracle.lcp_array(ss, want))


def test_one_repeated_character_closed_form_and_fast():
    """A text of 2^20 equal characters: suffix k of the sorted order is the one of
    length k + 1 (shorter suffixes are prefixes of longer ones), and its LCP with
    the previous one is k.  Direct string sorting would read n^2/2 characters;
    prefix doubling takes log2(n / 64) rounds."""
    m = sss()
    n = 1 << 20
    t = torch.full((n,), ord("A"), dtype=torch.uint8, device="cuda")
    m.sss_suffix_sort(t, 0)  # warm-up (work memory, module loading)
    m.context().sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sa, lcp = m.sss_suffix_sort(t, 0)
    e1.record()
    m.context().sync()
    ms = e0.elapsed_time(e1)
    k = np.arange(n, dtype=np.int64)
    assert np.array_equal(m.u32(sa).astype(np.int64), n - 1 - k)
    assert np.array_equal(m.u32(lcp).astype(np.int64), k)
    assert ms < 1000.0, f"{ms:.1f} ms"
