"""Pins for the oracle's partitioned pipeline (Sections 3 and 4).

* Local sorts against Python's sort of each partition.
* Regular sampling against the sample-density property (at most
  ceil(n_i/(v+1)) strings between consecutive local samples, appendix lemma on
  string-based sampling) and the sample count p*(v+1).
* Splitters: f_j = V[j(v+1)-1] of the sample sorted by Python.
* Buckets: every string of bucket j lies in (f_j, f_{j+1}] by Python's bytes
  order on the truncated strings; bucket sizes within the appendix bound
  (|V^j| + p) * ceil(omega) for unique strings.
* Merge and whole pipeline against Python's sort of the full set.
* Truncated order == full order for approx-truncated strings (Section 4 runs the
  merge sort on the approximated prefixes only).
"""
import math
import random

import numpy as np
import pytest

import datagen
import oracle
from test_oracle_sort import py_lcp, py_sort


def rand_strings(seed, n, unique=False):
    rnd = random.Random(seed)
    strs = []
    seen = set()
    prefixes = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 12))) for _ in range(5)]
    while len(strs) < n:
        s = rnd.choice(prefixes) + bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 10)))
        if unique and s in seen:
            continue
        seen.add(s)
        strs.append(s)
    return strs


@pytest.mark.parametrize("n,p", [(50, 1), (50, 3), (97, 8), (5, 8), (0, 2), (1, 1), (64, 16)])
def test_local_sort(n, p):
    strs = rand_strings(n + p, n)
    ss = datagen.from_strings(strs)
    rp, rl = oracle.local_sort(ss, p)
    for i in range(p):
        lo, hi = oracle.part_lo(n, p, i), oracle.part_lo(n, p, i + 1)
        part = strs[lo:hi]
        want = [lo + k for k in py_sort(part)]
        assert list(rp[lo:hi]) == want
        got_l = list(rl[lo:hi])
        assert got_l == py_lcp(strs, want)


@pytest.mark.parametrize("n,p,v", [(100, 4, 2), (1000, 16, 2), (37, 5, 3), (10, 10, 2), (7, 3, 1)])
def test_sampling_density_and_count(n, p, v):
    strs = rand_strings(n, n)
    ss = datagen.from_strings(strs)
    rp, _ = oracle.local_sort(ss, p)
    smp = oracle.samples(rp, n, p, v)
    nonempty = sum(1 for i in range(p) if oracle.part_lo(n, p, i + 1) > oracle.part_lo(n, p, i))
    assert smp.size == nonempty * (v + 1)
    pos = {int(x): r for r, x in enumerate(rp)}
    k = 0
    for i in range(p):
        lo, hi = oracle.part_lo(n, p, i), oracle.part_lo(n, p, i + 1)
        if hi == lo:
            continue
        ranks = [pos[int(s)] - lo for s in smp[k:k + v + 1]]
        k += v + 1
        omega = math.ceil((hi - lo) / (v + 1))
        prev = -1
        for r in ranks:
            assert 0 <= r < hi - lo
            assert r - prev - 1 <= omega  # strings strictly between consecutive samples
            prev = r
        assert ranks[-1] == hi - lo - 1


@pytest.mark.parametrize("seed,n,p", [(0, 200, 4), (1, 500, 8), (2, 64, 16), (3, 33, 5), (4, 3000, 16)])
def test_splitters_buckets_merge(seed, n, p):
    v = 2
    strs = rand_strings(seed, n, unique=True)
    ss = datagen.from_strings(strs)
    kmax = oracle.default_kmax(ss)
    res = oracle.pdms(ss, p, v, 0, kmax, seed)
    approx = res["approx"]
    tr = [s[: int(a)] for s, a in zip(strs, approx)]
    # sorted samples by Python on truncated strings (then index)
    smp = list(res["samples"])
    assert list(res["sorted_samples"]) == sorted(smp, key=lambda i: (tr[i], i))
    V = list(res["sorted_samples"])
    for j in range(1, p):
        k = (j * len(V)) // p - 1
        assert res["splitters"][j - 1] == (V[k] if k >= 0 else oracle.UINT32_MAX)
    # bucket membership: f_j < s <= f_{j+1} on truncated strings
    spl = [None] + [None if f == oracle.UINT32_MAX else tr[f] for f in res["splitters"]] + [None]
    bnd = res["bounds"]
    rp = res["run_perm"]
    sizes = [0] * p
    for i in range(p):
        lo = oracle.part_lo(n, p, i)
        for j in range(p):
            for q in range(lo + int(bnd[i, j]), lo + int(bnd[i, j + 1])):
                s = tr[rp[q]]
                if spl[j] is not None:
                    assert s > spl[j]
                if spl[j + 1] is not None:
                    assert s <= spl[j + 1]
                sizes[j] += 1
    # bucket bound from the appendix proof (general sizes): (|V^j| + p) * ceil(omega)
    maxni = max(oracle.part_lo(n, p, i + 1) - oracle.part_lo(n, p, i) for i in range(p))
    omega = math.ceil(maxni / (v + 1))
    for j in range(p):
        vj = sum(1 for x in V if (spl[j] is None or tr[x] > spl[j]) and (spl[j + 1] is None or tr[x] <= spl[j + 1]))
        assert sizes[j] <= (vj + p) * omega
    # merged output is the global sorted order with the full-string LCP array
    want = py_sort(strs)
    assert list(res["perm"]) == want
    assert list(res["lcp"]) == py_lcp(strs, want)


@pytest.mark.parametrize("seed", range(5))
def test_pipeline_with_duplicates_and_small_n(seed):
    rnd = random.Random(seed)
    strs = rand_strings(seed + 100, rnd.randint(1, 80))
    strs += [strs[rnd.randrange(len(strs))] for _ in range(len(strs) // 3)]  # duplicates
    rnd.shuffle(strs)
    ss = datagen.from_strings(strs)
    for p in [1, 2, 7, len(strs) + 3]:
        res = oracle.pdms(ss, p, 2, 0, oracle.default_kmax(ss), seed)
        want = py_sort(strs)
        assert list(res["perm"]) == want
        assert list(res["lcp"]) == py_lcp(strs, want)


def test_truncated_order_equals_full_order():
    ss = datagen.config1(count=3000)
    approx = oracle.doubling(ss, 0, 7, 4)
    full = oracle.sort(ss)
    trunc = oracle.sort_idx(ss, np.arange(ss.n), approx)
    assert (full == trunc).all()
    assert (oracle.lcp_array(ss, full) == oracle.lcp_array(ss, full, approx)).all()


def test_pdms_config2_scaled():
    ss = datagen.config2(n=4096)
    res = oracle.pdms(ss, 16, 2, 0, 9, 0)
    strs = ss.strings()
    want = py_sort(strs)
    assert list(res["perm"]) == want


# --- character-based sampling (Section 3.1.2; appendix "Character Based Sampling")

def skewed_strings(seed, n):
    """Lengths spread over two orders of magnitude, so string counts and character
    counts of a partition differ a lot."""
    rnd = random.Random(seed)
    out = []
    for _ in range(n):
        ln = rnd.choice([0, 1, 2, 3, 5, 8, 20, 60, 150])
        out.append(bytes(rnd.choice(b"ACGT") for _ in range(ln)))
    return out


def _char_case(seed, n, p, v):
    ss = datagen.from_strings(skewed_strings(seed, n))
    run_perm, _ = oracle.local_sort(ss, p)
    smp = oracle.samples_char(ss, run_perm, p, v)
    return ss, run_perm, smp


@pytest.mark.parametrize("seed,n,p,v", [(1, 60, 4, 2), (2, 200, 8, 2), (3, 97, 3, 5), (4, 40, 16, 1), (5, 7, 5, 2)])
def test_char_sampling_count_and_density(seed, n, p, v):
    ss, run_perm, smp = _char_case(seed, n, p, v)
    lens = ss.lens.astype(np.int64)
    N = int(lens.sum())
    if N == 0:
        return
    assert len(smp) == p * (v + 1)  # deficits are made up by the first partitions
    omega = N / (p * (v + 1))
    lmax = int(lens.max())
    sampled = set(int(s) for s in smp)
    # sample-density lemma: a contiguous piece of a run holding k sample strings
    # has at most (k+1)(omega + lmax) characters
    for i in range(p):
        lo, hi = oracle.part_lo(n, p, i), oracle.part_lo(n, p, i + 1)
        run = [int(x) for x in run_perm[lo:hi]]
        for a in range(len(run)):
            chars, k = 0, 0
            for b in range(a, len(run)):
                chars += int(lens[run[b]])
                k += run[b] in sampled
                assert chars <= (k + 1) * (omega + lmax) + 1e-9, (i, a, b)


@pytest.mark.parametrize("seed,n,p,v", [(11, 300, 4, 2), (12, 500, 8, 2), (13, 400, 8, 8), (14, 64, 16, 2)])
def test_char_sampling_bucket_bound(seed, n, p, v):
    """Every bucket holds at most (1 + p/v) N/p + (1 + (v+1)/p) p lmax characters
    (appendix theorem on character-based partitioning, r = p' = p)."""
    ss, run_perm, smp = _char_case(seed, n, p, v)
    lens = ss.lens.astype(np.int64)
    N, lmax = int(lens.sum()), int(lens.max())
    _, spl = oracle.splitters(ss, smp, p)
    bnd = oracle.bounds(ss, run_perm, p, spl).reshape(p, p + 1)
    bound = (1 + p / v) * N / p + (1 + (v + 1) / p) * p * lmax
    for j in range(p):
        chars = 0
        for i in range(p):
            lo = oracle.part_lo(n, p, i)
            for q in range(lo + int(bnd[i][j]), lo + int(bnd[i][j + 1])):
                chars += int(lens[run_perm[q]])
        assert chars <= bound + 1e-9, (j, chars, bound)
    # and the buckets still partition the sorted order: merge == Python's sort
    perm, lcp = oracle.merge(ss, run_perm, p, bnd.reshape(-1))
    assert [ss.string(int(x)) for x in perm] == sorted(ss.strings())


def test_char_sampling_positions_by_search():
    """Each sample is the string whose characters cover floor(t N / (p (v+1)))
    in its run's character array, found here by a prefix-sum search; the
    partitions that make up the deficit add their last string."""
    ss, run_perm, smp = _char_case(21, 150, 6, 3)
    p, v, n = 6, 3, 150
    lens = ss.lens.astype(np.int64)
    N, want = int(lens.sum()), p * (v + 1)
    exp, total = [], 0
    counts = []
    for i in range(p):
        lo, hi = oracle.part_lo(n, p, i), oracle.part_lo(n, p, i + 1)
        Ci = int(lens[run_perm[lo:hi]].sum())
        counts.append(max(0, -(-Ci * want // N) - 1))
    extra = max(0, want - sum(counts))
    for i in range(p):
        lo, hi = oracle.part_lo(n, p, i), oracle.part_lo(n, p, i + 1)
        if hi == lo:
            continue
        ends = np.cumsum(lens[run_perm[lo:hi]])
        for t in range(1, counts[i] + 1):
            x = t * N // want
            exp.append(int(run_perm[lo + int(np.searchsorted(ends, x, side="right"))]))
        if extra:
            exp.append(int(run_perm[hi - 1]))
            extra -= 1
    assert [int(s) for s in smp] == exp


def test_char_sampling_all_empty_falls_back():
    ss = datagen.from_strings([b""] * 20)
    run_perm, _ = oracle.local_sort(ss, 4)
    assert np.array_equal(oracle.samples_char(ss, run_perm, 4, 2), oracle.samples(run_perm, 20, 4, 2))
