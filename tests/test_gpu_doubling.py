"""Stage B on the GPU (prefix doubling) against the oracle's step-by-step
doubling, element by element through the C ABI (bit-exact: integer work)."""
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


def run_gpu(ss, p, kmin, kmax, seed, use_runs, sort_dedupe=False, per_round=False):
    m = sss()
    chars, offs, lens = m.to_device(ss)
    flags = (m.SSS_FLAG_DEDUPE_SORT if sort_dedupe else 0) | (m.SSS_FLAG_NO_CTA_ROUNDS if per_round else 0)
    prm = m.params(kmin=kmin, kmax=kmax, hash_seed=seed, flags=flags)
    if use_runs:
        rp, rl = m.sss_local_sort(chars, offs, lens, p)
        a = m.sss_dist_prefix(chars, offs, lens, rp, rl, p, prm)
    else:
        a = m.sss_dist_prefix(chars, offs, lens, None, None, 1, prm)
    m.context().sync()
    return u32(a)


def check(ss, p=1, kmin=0, kmax=None, seed=0):
    if kmax is None:
        kmax = oracle.default_kmax(ss)
    want = oracle.doubling(ss, kmin, kmax, seed)
    # hash table with rounds of few keys inside one CTA (the default), hash table
    # with per-round kernels only, sorted keys
    for use_runs in (False, True):
        for sort_dedupe, per_round in ((False, False), (False, True), (True, False)):
            got = run_gpu(ss, p, kmin, kmax, seed, use_runs, sort_dedupe, per_round)
            bad = np.flatnonzero(got != want)
            assert bad.size == 0, (f"use_runs={use_runs} sort_dedupe={sort_dedupe} per_round={per_round}: approx "
                                   f"differs at {bad[:5]} got {got[bad[:5]]} want {want[bad[:5]]}")


def test_handworked_example():
    strs = [b"CAB", b"CA", b"BBA", b"CAB", b"A", b"CABD", b"BBAC", b"CC"]
    ss = datagen.from_strings(strs)
    for p in (1, 2, 3, 8):
        check(ss, p, 0, 3)
    assert list(run_gpu(ss, 1, 0, 3, 0, False)) == [3, 2, 3, 3, 1, 4, 4, 2]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("kmin,kmax", [(0, 9), (2, 9), (0, 3), (4, 4), (5, 2)])
def test_random_sets(seed, kmin, kmax):
    rnd = random.Random(seed * 7 + kmin)
    strs = []
    pre = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 70))) for _ in range(4)]
    for _ in range(rnd.randint(1, 3000)):
        strs.append(rnd.choice(pre)[: rnd.randint(0, 70)] + bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 9))))
    ss = datagen.from_strings(strs)
    check(ss, rnd.choice([1, 3, 16]), kmin, kmax, seed)


def test_heavy_duplicates():
    rnd = random.Random(11)
    pool = [bytes(rnd.choice(b"AB") for _ in range(rnd.randint(0, 30))) for _ in range(6)]
    strs = [rnd.choice(pool) for _ in range(40000)]
    check(datagen.from_strings(strs), 4)


def test_config1():
    check(datagen.config1(), 1, 0, 7, 1)


def test_config2_scaled():
    check(datagen.config2(n=60000), 16, 0, 9, 0)


def test_suffixes_scaled():
    check(datagen.suffix_set(seed=3, text_len=1 << 15, n=1 << 13, max_len=256), 8)


@pytest.mark.parametrize("seed", [0, 12345, 2**63 + 5])
def test_hash_seeds(seed):
    check(datagen.config1(count=5000), 2, 0, 7, seed)
