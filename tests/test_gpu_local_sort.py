"""Stage A on the GPU (local sort with LCP output, exact dist) against the oracle,
element by element, through the C ABI.  Integer work: the bar is bit-exact."""
import random

import numpy as np
import pytest

import datagen
import oracle
from gpu_util import u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sss():
    import paper_2404_16517_gb300 as m
    return m


def check_plain(ss, check_dist=True):
    m = sss()
    chars, offs, lens = m.to_device(ss)
    perm, lcp, dist, _ = m.sss_sort(chars, offs, lens, 1, want_dist=check_dist)
    m.context().sync()
    want = oracle.sort(ss)
    got = u32(perm)
    assert np.array_equal(got, want), f"perm differs at {np.flatnonzero(got != want)[:5]}"
    wl = oracle.lcp_array(ss, want)
    gl = u32(lcp)
    assert np.array_equal(gl, wl), f"lcp differs at {np.flatnonzero(gl != wl)[:5]}"
    if check_dist:
        wd = oracle.dist(ss, want, wl)
        assert np.array_equal(u32(dist), wd)


def check_local(ss, p):
    m = sss()
    chars, offs, lens = m.to_device(ss)
    rp, rl = m.sss_local_sort(chars, offs, lens, p)
    m.context().sync()
    wp, wl = oracle.local_sort(ss, p)
    assert np.array_equal(u32(rp), wp)
    assert np.array_equal(u32(rl), wl)


def test_handworked_example():
    strs = [b"CAB", b"CA", b"BBA", b"CAB", b"A", b"CABD", b"BBAC", b"CC"]
    check_plain(datagen.from_strings(strs))


@pytest.mark.parametrize("strs", [
    [b"X"], [b"B", b"A"], [b"", b""], [b"", b"A", b""],
    [b"SAME"] * 100,
    [b""] * 50 + [b"A"] * 50,
    [b"A" * k for k in range(40, 0, -1)],
    [b"ABCDEFGH"[:k] for k in (7, 8, 9, 15, 16, 17) for _ in range(3)],
])
def test_edge_sets(strs):
    strs = [s if s else b"" for s in strs]
    ss = datagen.from_strings(strs)
    check_plain(ss)


def test_word_boundary_lengths():
    rnd = random.Random(1)
    strs = []
    for L in (7, 8, 9, 15, 16, 17, 23, 24, 25):
        base = bytes(rnd.choice(b"AB") for _ in range(L))
        for _ in range(20):
            k = rnd.randint(0, L)
            strs.append(base[:k] + bytes(rnd.choice(b"AB") for _ in range(rnd.randint(0, 3))))
    check_plain(datagen.from_strings(strs))


@pytest.mark.parametrize("n", [3, 60, 65, 700, 2048, 2049, 5000, 20000])
def test_long_common_prefixes(n):
    rnd = random.Random(n)
    pre = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.choice([0, 256, 300, 513]))) for _ in range(3)]
    strs = [rnd.choice(pre) + bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 12))) for _ in range(n)]
    check_plain(datagen.from_strings(strs))


def test_many_duplicates_large_segment():
    rnd = random.Random(5)
    pool = [bytes(rnd.choice(b"AB") for _ in range(rnd.randint(0, 20))) for _ in range(7)]
    strs = [rnd.choice(pool) for _ in range(30000)]
    check_plain(datagen.from_strings(strs))


def test_unaligned_overlapping_views():
    # suffix-like strings: views into one text at arbitrary offsets
    ss = datagen.suffix_set(seed=9, text_len=1 << 14, n=1 << 12, max_len=256)
    check_plain(ss)


def test_config1_full():
    check_plain(datagen.config1())


@pytest.mark.parametrize("p", [1, 2, 16, 37])
def test_local_sort_partitions(p):
    ss = datagen.config2(n=40000)
    check_local(ss, p)


def test_local_sort_more_partitions_than_strings():
    ss = datagen.from_strings([b"B", b"A", b"C"])
    check_local(ss, 8)


def test_dna_instances_mixed_lengths():
    sizes = np.array([64, 300, 2100, 9000], np.int64)
    ss, first = datagen.instance_set(4, sizes, 8, 300, np.array([0.1, 0.5, 0.9, 0.7]), datagen.DNA)
    check_plain(ss)


def test_empty_input():
    m = sss()
    chars = torch.zeros(1, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(0, dtype=torch.int64, device="cuda")
    lens = torch.zeros(0, dtype=torch.int32, device="cuda")
    perm, lcp, _, _ = m.sss_sort(chars, offs, lens, 1)
    m.context().sync()
    assert perm.numel() == 0


def test_checked_mode_flags_bad_input():
    m = sss()
    ss = datagen.from_strings([b"AB", b"CD"])
    chars, offs, lens = m.to_device(ss)
    bad_lens = torch.tensor([2, 9], dtype=torch.int32, device="cuda")  # runs past the chars array
    with pytest.raises(m.SssError) as ei:
        m.sss_sort(chars, offs, bad_lens, 1, prm=m.params(flags=m.SSS_FLAG_CHECKED))
    assert ei.value.status == 5
    # the context stays usable
    check_plain(ss)


@pytest.mark.parametrize("n,order", [(1500, "up"), (1500, "down"), (6000, "up"), (6000, "down")])
@pytest.mark.parametrize("knobs", [{}, {"cta_cap": 64, "direct_cap": 64, "bucket_target": 256}])
def test_nested_prefixes_in_length_order(n, order, knobs):
    """Strings A, AA, AAA, ... (each a prefix of the next) in length order: with
    the segment's first member as reference every round would peel off a few
    strings; a pseudo-random reference keeps the number of rounds logarithmic."""
    import time
    import paper_2404_16517_gb300 as m
    ks = list(range(1, n + 1))
    if order == "down":
        ks.reverse()
    ss = datagen.from_strings([b"A" * k for k in ks])
    chars, offs, lens = m.to_device(ss)
    t0 = time.time()
    perm, lcp, _, _ = m.sss_sort(chars, offs, lens, 1, m.params(**knobs))
    m.context().sync()
    assert time.time() - t0 < 30
    want = np.argsort(np.array(ks), kind="stable").astype(np.uint32)
    assert np.array_equal(m.u32(perm), want)
    sk = np.array(ks)[want]
    assert np.array_equal(m.u32(lcp), np.concatenate([[0], sk[:-1]]).astype(np.uint32))
