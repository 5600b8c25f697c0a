"""Seeded random cases through the whole path against the oracle: string
shapes (random DNA, template prefixes, nested prefixes, heavy duplicates,
length skew, very short), partition counts up to 300, every flag and random
tuning knobs; plus batches of random instance cuts.  Bit-exact perm, LCP and
dist."""
import random

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _strings(rnd):
    kind = rnd.choice(["dna", "templ", "nested", "dups", "skew", "short"])
    n = rnd.choice([1, 2, 3, 17, 100, 1000, 5000, 20000])
    if kind == "dna":
        return [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 40))) for _ in range(n)]
    if kind == "templ":
        T = [bytes(rnd.choice(b"AB") for _ in range(rnd.randint(0, 300))) for _ in range(rnd.randint(1, 8))]
        out = []
        for _ in range(n):
            t = rnd.choice(T)
            out.append(t[:rnd.randint(0, len(t))] + bytes(rnd.choice(b"AB") for _ in range(rnd.randint(0, 12))))
        return out
    if kind == "nested":
        base = bytes(rnd.choice(b"XY") for _ in range(1200))
        return [base[:rnd.randint(0, 1200)] for _ in range(n)]
    if kind == "dups":
        P = [bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 20))) for _ in range(rnd.randint(1, 30))]
        return [rnd.choice(P) for _ in range(n)]
    if kind == "skew":
        return [bytes(rnd.choice(b"ACGT") for _ in range(rnd.choice([1, 2, 500]) if rnd.random() < 0.1
                                                         else rnd.randint(0, 8))) for _ in range(n)]
    return [bytes(rnd.choice(b"AB") for _ in range(rnd.randint(0, 3))) for _ in range(n)]


@pytest.mark.parametrize("seed", range(6))
def test_fuzz(seed):
    import paper_2404_16517_gb300 as sss
    rnd = random.Random(1000 + seed)
    flag_set = (sss.SSS_FLAG_MS, sss.SSS_FLAG_DEDUPE_SORT, sss.SSS_FLAG_MERGE_TREE, sss.SSS_FLAG_CHAR_SAMPLING,
                sss.SSS_FLAG_GRAPH)
    for case in range(25):
        strs = _strings(rnd)
        ss = datagen.from_strings(strs)
        chars, offs, lens = sss.to_device(ss)
        p = rnd.choice([1, 1, 2, 3, 16, 64, 300])
        flags = 0
        for f in flag_set:
            if rnd.random() < 0.3:
                flags |= f
        knobs = {}
        if rnd.random() < 0.5:
            knobs = dict(cta_cap=rnd.choice([64, 100, 512, 2048]), direct_cap=rnd.choice([64, 1000, 8192]),
                         bucket_target=rnd.choice([256, 1000, 4096]), warp_cap=rnd.choice([2, 7, 32]))
        prm = sss.params(flags=flags, v=rnd.choice([1, 2, 5]), **knobs)
        want = oracle.sort(ss)
        wl = oracle.lcp_array(ss, want)
        perm, lcp, dist, _ = sss.sss_sort(chars, offs, lens, p, prm, want_dist=True)
        sss.context().sync()
        tag = (seed, case, len(strs), p, hex(flags), knobs)
        assert np.array_equal(sss.u32(perm), want), tag
        assert np.array_equal(sss.u32(lcp), wl), tag
        assert np.array_equal(sss.u32(dist), oracle.dist(ss, want, wl)), tag
        if len(strs) > 10 and rnd.random() < 0.4:
            cuts = sorted(rnd.sample(range(1, len(strs)), min(len(strs) - 1, rnd.randint(1, 30))))
            first = np.array([0] + cuts, dtype=np.uint64)
            sizes = np.diff(np.array([0] + cuts + [len(strs)])).astype(np.int64)
            bp, bl, _ = sss.sss_sort_batch(chars, offs, lens, first, sizes,
                                           sss.params(flags=flags & sss.SSS_FLAG_GRAPH, **knobs))
            sss.context().sync()
            BP, BL = sss.u32(bp), sss.u32(bl)
            for k in range(len(sizes)):
                a, b = int(first[k]), int(first[k]) + int(sizes[k])
                sub = datagen.StringSet(ss.chars, ss.offs[a:b], ss.lens[a:b])
                w = oracle.sort(sub)
                assert np.array_equal(BP[a:b], w), tag + (k,)
                assert np.array_equal(BL[a:b], oracle.lcp_array(sub, w)), tag + (k,)
