"""The allocation-free doubling entry point (for callers that cannot allocate
device memory: it keeps its state in a fixed device array inside libsss.so)
gives the same approximate distinguishing prefixes as sss_dist_prefix and as
the oracle, on two calls in a row (the second call must not see leftovers of
the first), for several round ranges: the default one, a finite kmax that
leaves strings unretired, a kmin >= 4 whose first round has no hash state to
resume from, and kmin > kmax (no rounds at all).

Collected last on purpose: if it fails, every other test has already run."""
import ctypes as C
import random

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sets():
    rnd = random.Random(5)
    pool = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 40))) for _ in range(50)]
    dups = [rnd.choice(pool) + bytes(rnd.choice(b"AC") for _ in range(rnd.randint(0, 3))) for _ in range(7000)]
    return [datagen.config1(count=20000), datagen.from_strings(dups),
            datagen.config2(n=4194304, count=65536)]


KRANGES = [(0, None), (0, 3), (5, None), (4, 2)]


def _call(m, chars, offs, lens, n, prm, out):
    return m.lib().sss_dist_prefix_noalloc(C.c_void_p(chars.data_ptr()), chars.numel(), C.c_void_p(offs.data_ptr()),
                                           C.c_void_p(lens.data_ptr()), n, C.byref(prm), C.c_void_p(out.data_ptr()),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("kr", KRANGES, ids=lambda k: f"k{k[0]}-{'auto' if k[1] is None else k[1]}")
@pytest.mark.parametrize("idx", [0, 1, 2])
def test_noalloc_matches_sss_dist_prefix_and_oracle_twice(idx, kr):
    import paper_2404_16517_gb300 as m
    ss = _sets()[idx]
    chars, offs, lens = m.to_device(ss)
    n = ss.n
    kmin, kmax = kr
    prm = m.params(kmin=kmin, kmax=m.SSS_KMAX_AUTO if kmax is None else kmax, hash_seed=7)
    want = m.sss_dist_prefix(chars, offs, lens, None, None, 1, prm)  # the allocating entry point
    m.context().sync()
    want = want.cpu().numpy().view(np.uint32)
    okmax = oracle.default_kmax(ss) if kmax is None else kmax
    want_oracle = oracle.doubling(ss, kmin, okmax, 7)
    assert np.array_equal(want, want_oracle), "sss_dist_prefix differs from the oracle"
    for call in range(2):
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st = _call(m, chars, offs, lens, n, prm, out)
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want_oracle), f"call {call}: differs at {np.flatnonzero(got != want_oracle)[:5]}"


def test_noalloc_binding_wrapper_matches_oracle():
    import paper_2404_16517_gb300 as m
    ss = _sets()[1]
    chars, offs, lens = m.to_device(ss)
    got = m.sss_dist_prefix_noalloc(chars, offs, lens, m.params(hash_seed=3))
    torch.cuda.synchronize()
    assert np.array_equal(m.u32(got), oracle.doubling(ss, 0, oracle.default_kmax(ss), 3))


def test_noalloc_rejects_too_many_strings():
    import paper_2404_16517_gb300 as m
    n = m.NOALLOC_MAX_STRINGS + 1
    chars = torch.full((n,), 65, dtype=torch.uint8, device="cuda")
    offs = torch.arange(n, dtype=torch.int64, device="cuda")
    lens = torch.ones(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = m.lib().sss_dist_prefix_noalloc(C.c_void_p(chars.data_ptr()), n, C.c_void_p(offs.data_ptr()),
                                         C.c_void_p(lens.data_ptr()), n, None, C.c_void_p(out.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1  # SSS_ERR_INVALID_ARG: beyond the fixed capacity, nothing enqueued
    with pytest.raises(ValueError):
        m.sss_dist_prefix_noalloc(chars, offs, lens)
