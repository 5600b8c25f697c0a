"""Suffix sorting through sss_suffix_sort (suffix views of one text, stage A):
the suffix array and LCP array equal Python's sort of the suffixes on small
texts (repetitive ones included) and the oracle's sort of the suffix views on a
Markov text, whole and truncated."""
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


CASES = [b"banana", b"A", b"AB", b"mississippi", b"A" * 1500, b"AB" * 900, b"ABC" * 400 + b"ABD",
         bytes(random.Random(1).choice(b"AC") for _ in range(3000)),
         bytes(random.Random(2).choice(b"ACGT") for _ in range(5000))]


@pytest.mark.parametrize("i", range(len(CASES)))
@pytest.mark.parametrize("max_len", [0, 7])
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
