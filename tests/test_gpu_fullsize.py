"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot sort 4.2M x 500 characters in seconds, so the outputs are
checked one by one instead: perm is a permutation; every adjacent pair is in
order (ties by index) with lcp equal to the oracle's pairwise LCP (a sorted,
tie-broken order is unique, so this fixes perm and lcp completely); dist is the
oracle's from that order; approx equals the doubling closed form
min(len, max(2^kmin, nextpow2(dist))) (len once nextpow2(dist) > 2^kmax), which
holds unless two different prefixes share a 64-bit key."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def nextpow2(a):
    a = np.maximum(a.astype(np.int64), 1)
    return (1 << np.ceil(np.log2(a)).astype(np.int64)).astype(np.int64)


def check_full(ss, perm, lcp, dist, approx, kmax):
    n = ss.n
    perm = perm.astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(n)), "perm is not a permutation"
    bad = oracle.check_sorted(ss, perm.astype(np.uint32), lcp)
    assert bad == n, f"order or lcp wrong at rank {bad}"
    assert np.array_equal(dist, oracle.dist(ss, perm.astype(np.uint32), lcp))
    d = dist.astype(np.int64)
    np2 = nextpow2(d)
    lens = ss.lens.astype(np.int64)
    want = np.where(np2 <= (1 << kmax), np.minimum(lens, np2), lens)
    assert np.array_equal(approx.astype(np.int64), want)


def test_config2_full_size_bench_configuration():
    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as m
    chars, offs, lens = dgc.config2()
    perm, lcp, dist, approx = m.sss_sort(chars, offs, lens, 16, want_dist=True, want_approx=True)
    m.context().sync()
    ss = datagen.StringSet(chars.cpu().numpy(), offs.cpu().numpy().view(np.uint64),
                           lens.cpu().numpy().view(np.uint32))
    check_full(ss, m.u32(perm), m.u32(lcp), m.u32(dist), m.u32(approx), 9)


def test_config3_full_size_suffixes():
    import paper_2404_16517_gb300 as m
    ss = datagen.config3()
    chars, offs, lens = m.to_device(ss)
    perm, lcp, dist, approx = m.sss_sort(chars, offs, lens, 64, want_dist=True, want_approx=True)
    m.context().sync()
    check_full(ss, m.u32(perm), m.u32(lcp), m.u32(dist), m.u32(approx), 8)


def test_config1_full_size_plain():
    import paper_2404_16517_gb300 as m
    ss = datagen.config1()
    chars, offs, lens = m.to_device(ss)
    perm, lcp, dist, _ = m.sss_sort(chars, offs, lens, 1, want_dist=True)
    m.context().sync()
    want = oracle.sort(ss)
    assert np.array_equal(m.u32(perm), want)
    assert np.array_equal(m.u32(lcp), oracle.lcp_array(ss, want))


def test_config4_full_size_batch():
    """All 4,096 instances (37.5M strings) in one batched call, every adjacent
    pair of every instance checked (order, ties by index, lcp)."""
    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as m
    chars, offs, lens, first = dgc.config4()
    sizes = np.diff(first).astype(np.int64)
    perm, lcp, _ = m.sss_sort_batch(chars, offs, lens, first[:-1], sizes)
    m.context().sync()
    P, L = m.u32(perm), m.u32(lcp)
    C, O, Ln = chars.cpu().numpy(), offs.cpu().numpy().view(np.uint64), lens.cpu().numpy().view(np.uint32)
    del chars, offs, lens
    for k in range(len(sizes)):
        a, b = int(first[k]), int(first[k + 1])
        sub = datagen.StringSet(C, O[a:b], Ln[a:b])
        p = P[a:b]
        assert np.array_equal(np.sort(p.astype(np.int64)), np.arange(b - a)), f"instance {k}: not a permutation"
        assert oracle.check_sorted(sub, p, L[a:b]) == b - a, f"instance {k}"


def test_largest_serving_request():
    """One request of the largest size (2^24 strings, about 8.5 GB) through the
    request loop, every adjacent pair checked."""
    import datagen.cuda as dgc
    from paper_2404_16517_gb300.serve import Request, Server
    n, seed, ratio = 1 << 24, 0x5EED5, 0.5
    tot = int(dgc.request_totals([seed], [n])[0])
    got = {}

    def grab(r):
        got["perm"] = r.perm.cpu().numpy().view(np.uint32).copy()
        got["lcp"] = r.lcp.cpu().numpy().view(np.uint32).copy()
        got["chars"] = srv.engine.arena[r._chars_off: r._chars_off + r.chars].cpu().numpy()

    srv = Server(budget_bytes=16 << 30, slots=1, on_done=grab)
    r = Request(rid=0, n=n, chars=tot, seed=seed, ratio=ratio)
    srv.run_closed_loop([r])
    srv.close()
    assert r.state == "done", r.error
    # the request's own table: regenerate offsets/lengths relative to its first character
    lens = torch.empty(n, dtype=torch.int32, device="cuda")
    offs = torch.empty(n, dtype=torch.int64, device="cuda")
    cp = torch.empty(n, dtype=torch.int32, device="cuda")
    sc = torch.empty(dgc.request_scratch_words(n), dtype=torch.int64, device="cuda")
    scratch_chars = torch.empty(tot, dtype=torch.uint8, device="cuda")
    dgc.request_into(scratch_chars, 0, offs, lens, cp, sc, seed, n, ratio)
    torch.cuda.synchronize()
    C = scratch_chars.cpu().numpy()
    assert np.array_equal(C, got["chars"]), "arena characters differ from the request's definition"
    ss = datagen.StringSet(C, offs.cpu().numpy().view(np.uint64), lens.cpu().numpy().view(np.uint32))
    assert np.array_equal(np.sort(got["perm"].astype(np.int64)), np.arange(n))
    assert oracle.check_sorted(ss, got["perm"], got["lcp"]) == n
