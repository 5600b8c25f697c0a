"""The all-core oracle pipeline (the CPU baseline) equals the single-threaded
one: same permutation, LCP array and approximate distinguishing prefixes, for
several thread counts and partition counts, duplicates and empty strings
included."""
import random

import numpy as np
import pytest

import datagen
import oracle


def _sets():
    rnd = random.Random(11)
    dna = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 24))) for _ in range(3000)]
    dna += dna[:500]  # duplicates
    return [datagen.config2(n=4194304, count=6000), datagen.config1(count=5000), datagen.from_strings(dna),
            datagen.from_strings([b"", b"A", b"", b"AB"])]


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("p", [1, 4, 16])
def test_parallel_pipeline_equals_serial(threads, p):
    for ss in _sets():
        want = oracle.pdms(ss, p, 2, 0, None, 5)
        perm, lcp, approx = oracle.pdms_parallel(ss, p, 2, 0, None, 5, nthreads=threads)
        assert np.array_equal(perm, want["perm"])
        assert np.array_equal(lcp, want["lcp"])
        assert np.array_equal(approx, want["approx"])
        # and the plain definition of the order
        assert np.array_equal(perm, oracle.sort(ss))
