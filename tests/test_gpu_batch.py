"""Batched sorting (sss_sort_batch) against the oracle per instance, and each
instance's result in the batch equal to its result alone (bit-exact)."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sss():
    import paper_2404_16517_gb300 as m
    return m


def view(ss, a, b):
    return datagen.StringSet(ss.chars, ss.offs[a:b], ss.lens[a:b])


def test_batch_matches_oracle_per_instance():
    m = sss()
    ss, first = datagen.config4(m=96, size_cap=3000)
    chars, offs, lens = m.to_device(ss)
    sizes = np.diff(first).astype(np.int64)
    perm, lcp, dist = m.sss_sort_batch(chars, offs, lens, first[:-1], sizes, want_dist=True)
    m.context().sync()
    P, L, D = m.u32(perm), m.u32(lcp), m.u32(dist)
    for k in range(len(sizes)):
        a, b = int(first[k]), int(first[k + 1])
        sub = view(ss, a, b)
        want = oracle.sort(sub)
        assert np.array_equal(P[a:b], want), f"instance {k}"
        wl = oracle.lcp_array(sub, want)
        assert np.array_equal(L[a:b], wl), f"instance {k} lcp"
        assert np.array_equal(D[a:b], oracle.dist(sub, want, wl)), f"instance {k} dist"


def test_batch_equals_each_instance_alone():
    m = sss()
    ss, first = datagen.config4(m=24, size_cap=20000)
    chars, offs, lens = m.to_device(ss)
    sizes = np.diff(first).astype(np.int64)
    perm, lcp, _ = m.sss_sort_batch(chars, offs, lens, first[:-1], sizes)
    m.context().sync()
    P, L = m.u32(perm), m.u32(lcp)
    for k in range(len(sizes)):
        a, b = int(first[k]), int(first[k + 1])
        p1, l1, _, _ = m.sss_sort(chars, offs[a:b].contiguous(), lens[a:b].contiguous(), 1)
        m.context().sync()
        assert np.array_equal(P[a:b], m.u32(p1)), f"instance {k}"
        assert np.array_equal(L[a:b], m.u32(l1)), f"instance {k} lcp"


def test_batch_edges_and_errors():
    m = sss()
    strs = [b"B", b"A", b"C", b"A", b"ZZ", b"Z", b"", b"Q"]
    ss = datagen.from_strings(strs)
    chars, offs, lens = m.to_device(ss)
    # instances: [0,3) [3,3) [3,6) [7,8); position 6 uncovered
    perm, lcp, _ = m.sss_sort_batch(chars, offs, lens, [0, 3, 3, 7], [3, 0, 3, 1])
    m.context().sync()
    P = m.u32(perm)
    assert list(P[0:3]) == [1, 0, 2]
    assert list(P[3:6]) == [0, 2, 1]
    assert P[7] == 0
    with pytest.raises(m.SssError):
        m.sss_sort_batch(chars, offs, lens, [0, 2], [3, 3])  # overlap


def test_device_instance_generator_identical():
    import datagen.cuda as dgc
    sizes, r = datagen.config4_sizes(4, 40)
    sizes = np.minimum(sizes, 700)
    c, o, l, first = dgc.instance_set(4, sizes, 8, 300, r)
    ss, first2 = datagen.instance_set(4, sizes, 8, 300, r)
    assert np.array_equal(first, first2)
    assert np.array_equal(c.cpu().numpy()[:ss.chars.size], ss.chars)
    assert np.array_equal(l.cpu().numpy().view(np.uint32), ss.lens)


def test_batch_of_short_instances_fills_both_short_classes():
    # instances of 2..33 strings over {a, b} with many duplicates: the 2..4
    # string instances go to the 4-lane class, 5..32 to the warp class (both
    # filling one shared array, from its two ends), 33 to the 64-thread CTA
    m = sss()
    rng = np.random.default_rng(17)
    strs, sizes = [], []
    for k in range(3000):
        c = 2 + k % 32
        sizes.append(c)
        for _ in range(c):
            ln = int(rng.integers(0, 12))
            strs.append(bytes(rng.choice(np.frombuffer(b"ab", dtype=np.uint8), ln).tolist()))
    ss = datagen.from_strings(strs)
    sizes = np.array(sizes, dtype=np.int64)
    first = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    chars, offs, lens = m.to_device(ss)
    perm, lcp, _ = m.sss_sort_batch(chars, offs, lens, first[:-1], sizes)
    m.context().sync()
    P, L = m.u32(perm), m.u32(lcp)
    for k in range(len(sizes)):
        a, b = int(first[k]), int(first[k + 1])
        sub = view(ss, a, b)
        want = oracle.sort(sub)
        assert np.array_equal(P[a:b], want), f"instance {k}"
        assert np.array_equal(L[a:b], oracle.lcp_array(sub, want)), f"instance {k} lcp"
