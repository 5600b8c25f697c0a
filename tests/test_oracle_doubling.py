"""Pins for the oracle's prefix hashing and prefix doubling (Section 4).

* SplitMix64 against its published outputs (tests/golden/splitmix64.txt).
* The mod-(2^61-1) multiply against exact integer arithmetic.
* Key structure: a key depends only on the tested prefix.
* The doubling result against its closed form: absent hash collisions a string
  retires in the first round L = 2^k >= 2^kmin with L >= dist (its L-prefix is
  unique, or L covers the whole string), so
      approx = min(len, max(2^kmin, nextpow2(dist)))   if nextpow2(dist) <= 2^kmax
      approx = len                                     otherwise,
  with dist taken from an all-pairs brute force or from Python's own sort.
* The invariant dist <= approx <= min(2*dist, len) (kmin = 0, kmax large).
The 64-bit key values themselves are pinned in test_oracle_hash.py.
"""
import os
import random

import numpy as np
import pytest

import datagen
import oracle
from test_oracle_sort import brute_dist, py_lcp, py_sort, read_golden

P61 = (1 << 61) - 1


def nextpow2(x):
    k = 1
    while k < x:
        k <<= 1
    return k


def closed_form(dist, lens, kmin, kmax):
    out = []
    for d, L in zip(dist, lens):
        t = max(1 << kmin, nextpow2(max(d, 1)))
        out.append(min(L, t) if nextpow2(max(d, 1)) <= (1 << kmax) and (1 << kmin) <= (1 << kmax) else L)
    return out


def py_dist(strs):
    perm = py_sort(strs)
    lcp = py_lcp(strs, perm)
    n = len(strs)
    d = [0] * n
    for r, i in enumerate(perm):
        m = max(lcp[r] if r > 0 else 0, lcp[r + 1] if r + 1 < n else 0)
        d[i] = min(len(strs[i]), m + 1)
    return d


def test_splitmix64_published_outputs():
    g = read_golden("splitmix64.txt")
    want = [int(x, 16) for x in g["seed0"]]
    gamma = 0x9E3779B97F4A7C15
    # the k-th output of the sequence started at state 0 is the "first output"
    # of the sequence started at state (k-1)*gamma
    got = [oracle.splitmix64_first((k * gamma) & ((1 << 64) - 1)) for k in range(3)]
    assert got == want
    # the generators' counter-based form reuses the same output function
    assert datagen.smix_int(gamma) == want[0]


def test_mulmod61_exact():
    rnd = random.Random(7)
    cases = [(0, 0), (1, P61 - 1), (P61 - 1, P61 - 1), (2, (1 << 60)), ((1 << 61) - 2, 3)]
    cases += [(rnd.randrange(P61), rnd.randrange(P61)) for _ in range(2000)]
    for a, b in cases:
        assert oracle.mulmod61(a, b) == (a * b) % P61


def test_hash_base_range():
    for seed in range(50):
        b = oracle.hash_base(seed)
        assert 2 <= b < P61 - 1


def test_key_depends_only_on_prefix():
    rnd = random.Random(3)
    for _ in range(200):
        L = rnd.randint(0, 40)
        base = bytes(rnd.choice(b"ACGT") for _ in range(L))
        l = rnd.randint(0, L)
        other = base[:l] + bytes(rnd.choice(b"XYZ") for _ in range(rnd.randint(0, 10)))
        ss = datagen.from_strings([base, other])
        assert oracle.prefix_key(ss, 0, l, 11) == oracle.prefix_key(ss, 1, l, 11)


def test_keys_of_distinct_prefixes_differ_exhaustively():
    # all strings over {A,B,C} up to length 6 (1093 strings), each hashed in full
    import itertools
    strs = [bytes(t) for L in range(0, 7) for t in itertools.product(b"ABC", repeat=L)]
    ss = datagen.from_strings(strs)
    keys = {oracle.prefix_key(ss, i, len(s), 5) for i, s in enumerate(strs)}
    assert len(keys) == len(strs)
    # same characters, different tested length: different keys (the length is
    # part of the key), e.g. "AB" vs "AB" padded to 3 is not the same prefix
    ss2 = datagen.from_strings([b"AB", b"AB\x41"])
    assert oracle.prefix_key(ss2, 0, 2, 5) != oracle.prefix_key(ss2, 1, 3, 5)


def test_handworked_doubling():
    g = read_golden("handworked_example.txt")
    strs = [s.encode() for s in g["strings"]]
    ss = datagen.from_strings(strs)
    approx = oracle.doubling(ss, 0, 3, 0)
    assert list(approx) == [int(x) for x in g["approx"]]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("kmin,kmax", [(0, 6), (2, 6), (0, 2), (3, 3)])
def test_closed_form_random(seed, kmin, kmax):
    rnd = random.Random(seed * 31 + kmin)
    strs = []
    for _ in range(rnd.randint(1, 250)):
        L = rnd.choice([0, 1, 3, 8, 9, rnd.randint(0, 50)])
        strs.append(bytes(rnd.choice(b"AB" if seed % 2 else b"ACGT") for _ in range(L)))
    # plant shared prefixes and duplicates
    for _ in range(len(strs) // 4):
        i, j = rnd.randrange(len(strs)), rnd.randrange(len(strs))
        strs[j] = strs[i][: rnd.randint(0, len(strs[i]))] + strs[j]
    ss = datagen.from_strings(strs)
    d = brute_dist(strs) if len(strs) < 120 else py_dist(strs)
    approx = oracle.doubling(ss, kmin, kmax, seed)
    assert list(approx) == closed_form(d, [len(s) for s in strs], kmin, kmax)


def test_closed_form_config1_sample():
    ss = datagen.config1(count=4000)
    strs = ss.strings()
    d = py_dist(strs)
    approx, rounds = oracle.doubling(ss, 0, 7, 1, want_rounds=True)
    assert list(approx) == closed_form(d, [len(s) for s in strs], 0, 7)
    # bounds on the approximation (Section 4: approx >= dist)
    a = np.array(approx, np.int64)
    dd = np.array(d, np.int64)
    assert (a >= dd).all() and (a <= np.minimum(2 * dd, 100)).all()
    # active strings only shrink from round to round
    r = [int(x) for x in rounds if x]
    assert r == sorted(r, reverse=True) and r[0] == ss.n


def test_doubling_empty_and_duplicates():
    strs = [b"", b"", b"A", b"A", b"AB", b"AB", b"ABC"]
    ss = datagen.from_strings(strs)
    approx = oracle.doubling(ss, 0, 4, 9)
    assert list(approx) == [0, 0, 1, 1, 2, 2, 3]
