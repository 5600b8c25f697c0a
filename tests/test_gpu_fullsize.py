"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot sort 4.2M x 500 characters in seconds, so the outputs are
checked one by one instead: perm is a permutation; every adjacent pair is in
order (ties by index) with lcp equal to the oracle's pairwise LCP (a sorted,
tie-broken order is unique, so this fixes perm and lcp completely); dist is the
oracle's from that order; approx equals the doubling closed form
min(len, max(2^kmin, nextpow2(dist))) (len once nextpow2(dist) > 2^kmax), which
holds unless two different prefixes share a 64-bit key."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def nextpow2(a):
    a = np.maximum(a.astype(np.int64), 1)
    return (1 << np.ceil(np.log2(a)).astype(np.int64)).astype(np.int64)


def check_full(ss, perm, lcp, dist, approx, kmax):
    n = ss.n
    perm = perm.astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(n)), "perm is not a permutation"
    bad = oracle.check_sorted(ss, perm.astype(np.uint32), lcp)
    assert bad == n, f"order or lcp wrong at rank {bad}"
    assert np.array_equal(dist, oracle.dist(ss, perm.astype(np.uint32), lcp))
    d = dist.astype(np.int64)
    np2 = nextpow2(d)
    lens = ss.lens.astype(np.int64)
    want = np.where(np2 <= (1 << kmax), np.minimum(lens, np2), lens)
    assert np.array_equal(approx.astype(np.int64), want)


def test_config2_full_size_bench_configuration():
    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as m
    chars, offs, lens = dgc.config2()
    perm, lcp, dist, approx = m.sss_sort(chars, offs, lens, 16, want_dist=True, want_approx=True)
    m.context().sync()
    ss = datagen.StringSet(chars.cpu().numpy(), offs.cpu().numpy().view(np.uint64),
                           lens.cpu().numpy().view(np.uint32))
    check_full(ss, m.u32(perm), m.u32(lcp), m.u32(dist), m.u32(approx), 9)


def test_config3_full_size_suffixes():
    import paper_2404_16517_gb300 as m
    ss = datagen.config3()
    chars, offs, lens = m.to_device(ss)
    perm, lcp, dist, approx = m.sss_sort(chars, offs, lens, 64, want_dist=True, want_approx=True)
    m.context().sync()
    check_full(ss, m.u32(perm), m.u32(lcp), m.u32(dist), m.u32(approx), 8)


def test_config1_full_size_plain():
    import paper_2404_16517_gb300 as m
    ss = datagen.config1()
    chars, offs, lens = m.to_device(ss)
    perm, lcp, dist, _ = m.sss_sort(chars, offs, lens, 1, want_dist=True)
    m.context().sync()
    want = oracle.sort(ss)
    assert np.array_equal(m.u32(perm), want)
    assert np.array_equal(m.u32(lcp), oracle.lcp_array(ss, want))
