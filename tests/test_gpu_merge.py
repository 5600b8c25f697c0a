"""Stages C and D and the whole path on the GPU against the oracle: splitters
and bucket bounds, the LCP-compressed exchange + LCP merge, and sss_sort with
p > 1 (PDMS), element by element (bit-exact)."""
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


def rand_set(seed, n, dups=True):
    rnd = random.Random(seed)
    pre = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 40))) for _ in range(5)]
    strs = [rnd.choice(pre)[: rnd.randint(0, 40)] + bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 8)))
            for _ in range(n)]
    if dups:
        strs += [strs[rnd.randrange(n)] for _ in range(n // 5)] if n else []
        rnd.shuffle(strs)
    return datagen.from_strings(strs)


@pytest.mark.parametrize("seed,n,p", [(0, 500, 4), (1, 3000, 16), (2, 40, 7), (3, 5, 9), (4, 20000, 16)])
def test_partition_matches_oracle(seed, n, p):
    m = sss()
    ss = rand_set(seed, n)
    rp, _ = oracle.local_sort(ss, p)
    approx = oracle.doubling(ss, 0, oracle.default_kmax(ss), 0)
    _, want_spl = oracle.splitters(ss, oracle.samples(rp, ss.n, p, 2), p, approx)
    want_b = oracle.bounds(ss, rp, p, want_spl, approx)
    chars, offs, lens = m.to_device(ss)
    t_rp = torch.from_numpy(rp.view(np.int32)).cuda()
    t_tr = torch.from_numpy(approx.view(np.int32)).cuda()
    spl, bnd = m.sss_partition(chars, offs, lens, t_rp, p, trunc=t_tr)
    m.context().sync()
    assert np.array_equal(u32(spl), want_spl)
    assert np.array_equal(u32(bnd), want_b)


@pytest.mark.parametrize("tree", [False, True])
@pytest.mark.parametrize("seed,n,p,trunc", [(0, 800, 4, False), (1, 5000, 16, True), (2, 3000, 5, True),
                                            (3, 30000, 16, False), (4, 7, 3, True), (5, 60000, 2, True),
                                            (6, 40000, 256, True), (7, 30000, 255, False), (8, 20000, 100, True)])
def test_lcp_merge_matches_oracle(seed, n, p, trunc, tree):
    m = sss()
    ss = rand_set(seed, n)
    rp, rl = oracle.local_sort(ss, p)
    tr = oracle.doubling(ss, 0, oracle.default_kmax(ss), 0) if trunc else None
    _, spl = oracle.splitters(ss, oracle.samples(rp, ss.n, p, 2), p, tr)
    bnd = oracle.bounds(ss, rp, p, spl, tr)
    want_p, want_l = oracle.merge(ss, rp, p, bnd, tr)
    chars, offs, lens = m.to_device(ss)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    prm = m.params(flags=m.SSS_FLAG_MERGE_TREE if tree else 0)
    op, ol = m.sss_lcp_merge(chars, offs, lens, t(rp), t(rl), p, trunc=None if tr is None else t(tr), prm=prm)
    m.context().sync()
    assert np.array_equal(u32(op), want_p)
    assert np.array_equal(u32(ol), want_l)


def test_merge_many_equal_strings_oversized_sub_buckets():
    # 30000 strings from 3 values: sub-buckets of equal strings exceed one CTA
    rnd = random.Random(21)
    pool = [b"GATTACA" * 3, b"GATTACA" * 3 + b"T", b"CAT"]
    check_sort(datagen.from_strings([rnd.choice(pool) for _ in range(30000)]), 4)


def check_sort(ss, p, flags=0):
    m = sss()
    chars, offs, lens = m.to_device(ss)
    kmax = oracle.default_kmax(ss)
    perm, lcp, dist, approx = m.sss_sort(chars, offs, lens, p, prm=m.params(flags=flags), want_dist=True,
                                         want_approx=True)
    m.context().sync()
    want = oracle.sort(ss)
    gp = u32(perm)
    assert np.array_equal(gp, want), f"perm differs at {np.flatnonzero(gp != want)[:5]}"
    wl = oracle.lcp_array(ss, want)
    gl = u32(lcp)
    assert np.array_equal(gl, wl), f"lcp differs at {np.flatnonzero(gl != wl)[:5]}"
    assert np.array_equal(u32(dist), oracle.dist(ss, want, wl))
    wa = ss.lens if flags & m.SSS_FLAG_MS else oracle.doubling(ss, 0, kmax, 0)
    assert np.array_equal(u32(approx), wa)


@pytest.mark.parametrize("p", [2, 3, 16, 64])
def test_pdms_config2_scaled(p):
    check_sort(datagen.config2(n=50000), p)


def test_pdms_suffixes_scaled():
    check_sort(datagen.suffix_set(seed=3, text_len=1 << 16, n=1 << 15, max_len=256), 64)


@pytest.mark.parametrize("seed", range(4))
def test_pdms_random_with_duplicates(seed):
    rnd = random.Random(seed)
    check_sort(rand_set(seed + 50, rnd.randint(1, 4000)), rnd.choice([2, 5, 16]))


def test_pdms_more_partitions_than_strings():
    check_sort(datagen.from_strings([b"CAB", b"CA", b"BBA", b"CAB", b"A"]), 8)


def test_ms_mode_full_strings():
    m = sss()
    check_sort(datagen.config2(n=20000), 16, m.SSS_FLAG_MS)


def test_pdms_tree_merge_path():
    m = sss()
    check_sort(datagen.config2(n=30000), 16, m.SSS_FLAG_MERGE_TREE)


def test_pdms_many_partitions_tree_fallback():
    # p > 256 takes the pairwise-tree merge
    check_sort(rand_set(77, 6000), 300)


def test_pdms_config1():
    check_sort(datagen.config1(), 16)
