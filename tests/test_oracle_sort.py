"""Pins for the oracle's sort, LCP array and distinguishing prefixes.

The oracle (plain C) is checked against things other than itself: Python's own
bytes ordering (a library routine), os.path.commonprefix, an all-pairs brute
force for dist, exhaustive tiny inputs, and the hand-worked example of
tests/golden/handworked_example.txt (definitions of Section 2).
"""
import itertools
import os
import random

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            rows[k] = v
    return rows


def py_sort(strs):
    return sorted(range(len(strs)), key=lambda i: (strs[i], i))


def py_lcp(strs, perm):
    out = [0] * len(perm)
    for r in range(1, len(perm)):
        out[r] = len(os.path.commonprefix([strs[perm[r - 1]], strs[perm[r]]]))
    return out


def brute_dist(strs):
    """dist(s) = min(len s, 1 + max over all other strings t of lcp(s, t)),
    computed over all pairs (no sorting involved)."""
    n = len(strs)
    out = []
    for i in range(n):
        m = 0
        for j in range(n):
            if j != i:
                m = max(m, len(os.path.commonprefix([strs[i], strs[j]])))
        out.append(min(len(strs[i]), 1 + m) if n > 1 else min(len(strs[i]), 1))
    return out


def check_set(strs):
    ss = datagen.from_strings(strs)
    perm = oracle.sort(ss)
    assert list(perm) == py_sort(strs)
    lcp = oracle.lcp_array(ss, perm)
    assert list(lcp) == py_lcp(strs, list(perm))
    d = oracle.dist(ss, perm, lcp)
    assert list(d) == brute_dist(strs)
    assert oracle.check_sorted(ss, perm, lcp) == len(strs)


def test_handworked_example():
    g = read_golden("handworked_example.txt")
    strs = [s.encode() for s in g["strings"]]
    ss = datagen.from_strings(strs)
    perm = oracle.sort(ss)
    assert list(perm) == [int(x) for x in g["perm"]]
    lcp = oracle.lcp_array(ss, perm)
    assert list(lcp) == [int(x) for x in g["lcp"]]
    assert list(oracle.dist(ss, perm, lcp)) == [int(x) for x in g["dist"]]


def test_exhaustive_tiny_multisets():
    # every multiset of 1..4 strings over {A,B} of length <= 3 (with repeats)
    alphabet = [b""] + [bytes(t) for L in range(1, 4) for t in itertools.product(b"AB", repeat=L)]
    count = 0
    for m in range(1, 5):
        for combo in itertools.combinations_with_replacement(range(len(alphabet)), m):
            strs = [alphabet[c] for c in combo]
            # several orders of the same multiset
            rnd = random.Random(count)
            for _ in range(2):
                rnd.shuffle(strs)
                check_set(list(strs))
            count += 1
    assert count > 1000


@pytest.mark.parametrize("seed", range(6))
def test_random_sets(seed):
    rnd = random.Random(seed)
    strs = []
    for _ in range(rnd.randint(0, 300)):
        L = rnd.choice([0, 1, 2, 7, 8, 9, 15, 16, 17, rnd.randint(0, 40)])
        strs.append(bytes(rnd.choice(b"ACGT" if seed % 2 else b"AB") for _ in range(L)))
    if len(strs) > 1:
        check_set(strs)


def test_config1_sample_against_python():
    ss = datagen.config1(count=3000)
    strs = ss.strings()
    perm = oracle.sort(ss)
    assert list(perm) == py_sort(strs)
    lcp = oracle.lcp_array(ss, perm)
    assert list(lcp) == py_lcp(strs, list(perm))


def test_check_sorted_catches_planted_mistakes():
    ss = datagen.config1(count=500)
    perm = oracle.sort(ss)
    lcp = oracle.lcp_array(ss, perm)
    assert oracle.check_sorted(ss, perm, lcp) == ss.n
    bad = perm.copy()
    bad[10], bad[11] = bad[11], bad[10]
    assert oracle.check_sorted(ss, bad, lcp) == 11
    badl = lcp.copy()
    badl[200] += 1
    assert oracle.check_sorted(ss, perm, badl) == 200
    badl = lcp.copy()
    badl[0] = 1
    assert oracle.check_sorted(ss, perm, badl) == 0


def test_equal_strings_ordered_by_index():
    strs = [b"XY", b"XY", b"X", b"XY", b"", b""]
    ss = datagen.from_strings(strs)
    perm = oracle.sort(ss)
    assert list(perm) == [4, 5, 2, 0, 1, 3]
    lcp = oracle.lcp_array(ss, perm)
    assert list(lcp) == [0, 0, 0, 1, 2, 2]
    assert list(oracle.dist(ss, perm, lcp)) == [2, 2, 1, 2, 0, 0]


def test_truncated_compare():
    strs = [b"ABCD", b"ABCE", b"ABX"]
    ss = datagen.from_strings(strs)
    trunc = np.array([3, 3, 3], np.uint32)
    # truncated to 3 chars the first two are equal strings: index order
    assert oracle.cmp(ss, 0, 1, trunc) == -1
    assert oracle.cmp(ss, 1, 0, trunc) == 1
    assert oracle.lcp_pair(ss, 0, 1, trunc) == 3
    assert oracle.lcp_pair(ss, 0, 1) == 3
    assert oracle.cmp(ss, 1, 0) == 1
    assert list(oracle.sort_idx(ss, [2, 1, 0], trunc)) == [0, 1, 2]


def test_oracle_sorts_suffix_views_like_python():
    """Suffix views of one text (strings overlapping in the character array):
    the oracle's order equals Python's sort of the suffixes."""
    import random as _r
    for seed in range(4):
        rnd = _r.Random(seed)
        text = bytes(rnd.choice(b"AB") for _ in range(rnd.randint(1, 200)))
        n = len(text)
        offs = np.arange(n, dtype=np.uint64)
        ss = datagen.StringSet(np.frombuffer(text, np.uint8).copy(), offs, (n - offs).astype(np.uint32))
        want = sorted(range(n), key=lambda i: text[i:])
        assert list(oracle.sort(ss)) == want
