"""Tuning knobs change speed, never results: the batched and the full-pipeline
sorts give bit-identical outputs (and the oracle's) under extreme settings; the
autotuner returns one of its candidates."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXTREMES = [
    {},
    {"cta_cap": 64, "direct_cap": 64, "bucket_target": 256, "warp_cap": 2},
    {"cta_cap": 300, "direct_cap": 1000, "bucket_target": 4096, "warp_cap": 7},
    {"cta_cap": 2048, "direct_cap": 2048, "bucket_target": 777, "warp_cap": 32, "merge_ms": 8},
    {"cta_cap": 100000, "direct_cap": 1, "bucket_target": 1, "warp_cap": 1000},  # clamped
]


def test_batch_results_independent_of_knobs():
    import paper_2404_16517_gb300 as sss
    ss, first = datagen.config4(m=40, size_cap=20000)
    chars, offs, lens = sss.to_device(ss)
    sizes = np.diff(first).astype(np.int64)
    ref = None
    for k in EXTREMES:
        perm, lcp, _ = sss.sss_sort_batch(chars, offs, lens, first[:-1], sizes, sss.params(**k))
        sss.context().sync()
        got = (sss.u32(perm), sss.u32(lcp))
        if ref is None:
            ref = got
            for i in range(0, len(sizes), 7):  # a few instances against the oracle
                a, b = int(first[i]), int(first[i + 1])
                sub = datagen.StringSet(ss.chars, ss.offs[a:b], ss.lens[a:b])
                want = oracle.sort(sub)
                assert np.array_equal(got[0][a:b], want)
                assert np.array_equal(got[1][a:b], oracle.lcp_array(sub, want))
        else:
            assert np.array_equal(got[0], ref[0]), k
            assert np.array_equal(got[1], ref[1]), k


def test_pdms_results_independent_of_knobs():
    import paper_2404_16517_gb300 as sss
    ss = datagen.config2(n=1 << 15)
    chars, offs, lens = sss.to_device(ss)
    want = oracle.sort(ss)
    wl = oracle.lcp_array(ss, want)
    for k in EXTREMES:
        perm, lcp, _, _ = sss.sss_sort(chars, offs, lens, 8, sss.params(**k))
        sss.context().sync()
        assert np.array_equal(sss.u32(perm), want), k
        assert np.array_equal(sss.u32(lcp), wl), k


def test_autotuner_picks_a_candidate():
    import paper_2404_16517_gb300 as sss
    from paper_2404_16517_gb300 import autotune
    ss, first = datagen.config4(m=64, size_cap=10000)
    chars, offs, lens = sss.to_device(ss)
    sizes = np.diff(first).astype(np.int64)
    grid = {"cta_cap": [1024, 2048], "warp_cap": [16, 32]}
    best, table = autotune.tune_batch(chars, offs, lens, first[:-1], sizes, grid=grid, max_strings=1 << 16, reps=2)
    assert best in autotune.candidates(grid)
    assert len(table) == 4 and table[0][1] == best
    assert all(table[i][0] <= table[i + 1][0] for i in range(3))


def test_graph_round_loop_identical_and_reused():
    """SSS_FLAG_GRAPH runs the round loop as one graph launch: outputs identical
    to the host-driven loop, on a first call (capture), a repeated call (the
    kept graph) and a call with other inputs (a new capture)."""
    import paper_2404_16517_gb300 as sss
    G = sss.SSS_FLAG_GRAPH
    for m_inst, cap in ((40, 20000), (25, 9000)):
        ss, first = datagen.config4(m=m_inst, size_cap=cap)
        chars, offs, lens = sss.to_device(ss)
        sizes = np.diff(first).astype(np.int64)
        ref = sss.sss_sort_batch(chars, offs, lens, first[:-1], sizes, sss.params())
        for k in ({}, {"bucket_target": 4096, "cta_cap": 300}):
            for _ in range(2):
                got = sss.sss_sort_batch(chars, offs, lens, first[:-1], sizes, sss.params(flags=G, **k))
                sss.context().sync()
                assert np.array_equal(sss.u32(got[0]), sss.u32(ref[0])), k
                assert np.array_equal(sss.u32(got[1]), sss.u32(ref[1])), k
    ss = datagen.config2(n=1 << 15)
    chars, offs, lens = sss.to_device(ss)
    want = oracle.sort(ss)
    perm, lcp, _, _ = sss.sss_sort(chars, offs, lens, 8, sss.params(flags=G))
    sss.context().sync()
    assert np.array_equal(sss.u32(perm), want)
    assert np.array_equal(sss.u32(lcp), oracle.lcp_array(ss, want))
