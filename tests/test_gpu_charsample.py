"""Character-based regular sampling (Section 3.1.2, SSS_FLAG_CHAR_SAMPLING)
through the C ABI: splitters and bucket bounds bit-exact against the oracle, the
whole pipeline's output unchanged, and the buckets' character counts within the
appendix bound."""
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


def skewed(seed, n, maxlen=300):
    rnd = random.Random(seed)
    out = []
    templ = bytes(rnd.choice(b"ACGT") for _ in range(maxlen))
    for _ in range(n):
        ln = int(min(maxlen, rnd.expovariate(1 / 30))) if rnd.random() < 0.9 else rnd.randint(0, maxlen)
        cp = rnd.randint(0, ln)
        out.append(templ[:cp] + bytes(rnd.choice(b"ACGT") for _ in range(ln - cp)))
    return datagen.from_strings(out)


@pytest.mark.parametrize("seed,n,p,v,trunc", [(0, 3000, 4, 2, False), (1, 20000, 16, 2, True), (2, 500, 7, 5, True),
                                               (3, 5, 8, 2, False), (4, 40000, 32, 2, True), (5, 64, 2, 1, False)])
def test_char_partition_matches_oracle(seed, n, p, v, trunc):
    m = sss()
    ss = skewed(seed, n)
    rp, _ = oracle.local_sort(ss, p)
    tr = oracle.doubling(ss, 0, oracle.default_kmax(ss), 0) if trunc else None
    smp = oracle.samples_char(ss, rp, p, v, tr)
    _, want_spl = oracle.splitters(ss, smp, p, tr)
    want_b = oracle.bounds(ss, rp, p, want_spl, tr)
    chars, offs, lens = m.to_device(ss)
    t_rp = torch.from_numpy(rp.view(np.int32)).cuda()
    t_tr = torch.from_numpy(tr.view(np.int32)).cuda() if trunc else None
    spl, bnd = m.sss_partition(chars, offs, lens, t_rp, p, trunc=t_tr,
                               prm=m.params(v=v, flags=m.SSS_FLAG_CHAR_SAMPLING))
    m.context().sync()
    assert np.array_equal(m.u32(spl), want_spl)
    assert np.array_equal(m.u32(bnd).reshape(-1), want_b.reshape(-1))


def test_char_partition_all_empty_strings():
    m = sss()
    ss = datagen.from_strings([b""] * 50)
    rp, _ = oracle.local_sort(ss, 4)
    _, want_spl = oracle.splitters(ss, oracle.samples_char(ss, rp, 4, 2), 4)
    chars, offs, lens = m.to_device(ss)
    spl, bnd = m.sss_partition(chars, offs, lens, torch.from_numpy(rp.view(np.int32)).cuda(), 4,
                               prm=m.params(flags=m.SSS_FLAG_CHAR_SAMPLING))
    m.context().sync()
    assert np.array_equal(m.u32(spl), want_spl)


@pytest.mark.parametrize("tree", [False, True])
def test_char_sampling_pipeline_output_and_balance(tree):
    m = sss()
    ss = skewed(7, 60000, maxlen=1000)
    p, v = 16, 2
    want = oracle.sort(ss)
    flags = m.SSS_FLAG_CHAR_SAMPLING | (m.SSS_FLAG_MERGE_TREE if tree else 0)
    chars, offs, lens = m.to_device(ss)
    perm, lcp, _, approx = m.sss_sort(chars, offs, lens, p, m.params(flags=flags), want_approx=True)
    m.context().sync()
    assert np.array_equal(m.u32(perm), want)
    assert np.array_equal(m.u32(lcp), oracle.lcp_array(ss, want))
    # the oracle pipeline with character-based sampling: same approx, and its
    # buckets hold at most (1 + p/v) N/p + (1 + (v+1)/p) p lmax characters
    o = oracle.pdms(ss, p, v, char_sampling=True)
    assert np.array_equal(m.u32(approx), o["approx"])
    tl = o["approx"].astype(np.int64)
    N, lmax = int(tl.sum()), int(tl.max())
    bnd = o["bounds"].reshape(p, p + 1)
    for j in range(p):
        c = 0
        for i in range(p):
            lo = oracle.part_lo(ss.n, p, i)
            c += int(tl[o["run_perm"][lo + int(bnd[i][j]): lo + int(bnd[i][j + 1])]].sum())
        assert c <= (1 + p / v) * N / p + (1 + (v + 1) / p) * p * lmax
