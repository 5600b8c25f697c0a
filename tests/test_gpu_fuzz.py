"""Seeded random cases through the whole path against the oracle: string
shapes (random DNA, template prefixes, nested prefixes, heavy duplicates,
length skew, very short), partition counts up to 300, every flag, random hash
seeds and tuning knobs; plus batches of random instance cuts and the
host-input path.  Bit-exact perm, LCP, dist and (prefix doubling) approx.
SSS_FUZZ_SEEDS sets the number of seeds (25 cases each; default 6)."""
import os
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


def _host_sort(sss, ss, p, prm):
    h_chars = torch.from_numpy(ss.chars if ss.chars.size else np.zeros(1, np.uint8)).pin_memory()
    h_offs = torch.from_numpy(ss.offs.view(np.int64)).pin_memory()
    h_lens = torch.from_numpy(ss.lens.view(np.int32)).pin_memory()
    d_chars = torch.empty(h_chars.numel(), dtype=torch.uint8, device="cuda")
    d_offs = torch.empty(ss.n, dtype=torch.int64, device="cuda")
    d_lens = torch.empty(ss.n, dtype=torch.int32, device="cuda")
    h_perm = torch.full((ss.n,), -1, dtype=torch.int32).pin_memory()
    h_lcp = torch.full((ss.n,), -1, dtype=torch.int32).pin_memory()
    sss.sss_sort_host(h_chars, h_offs, h_lens, p, d_chars, d_offs, d_lens, prm, h_out_perm=h_perm, h_out_lcp=h_lcp)
    sss.context().sync()
    return h_perm.numpy().view(np.uint32), h_lcp.numpy().view(np.uint32)


@pytest.mark.parametrize("seed", range(int(os.environ.get("SSS_FUZZ_SEEDS", "6"))))
def test_fuzz(seed):
    import paper_2404_16517_gb300 as sss
    rnd = random.Random(1000 + seed)
    flag_set = (sss.SSS_FLAG_MS, sss.SSS_FLAG_DEDUPE_SORT, sss.SSS_FLAG_MERGE_TREE, sss.SSS_FLAG_CHAR_SAMPLING,
                sss.SSS_FLAG_GRAPH, sss.SSS_FLAG_NO_CTA_ROUNDS)
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
        hseed = rnd.randint(0, (1 << 31) - 1)
        prm = sss.params(flags=flags, v=rnd.choice([1, 2, 5]), hash_seed=hseed, **knobs)
        want = oracle.sort(ss)
        wl = oracle.lcp_array(ss, want)
        perm, lcp, dist, approx = sss.sss_sort(chars, offs, lens, p, prm, want_dist=True, want_approx=True)
        sss.context().sync()
        tag = (seed, case, len(strs), p, hex(flags), hseed, knobs)
        assert np.array_equal(sss.u32(perm), want), tag
        assert np.array_equal(sss.u32(lcp), wl), tag
        assert np.array_equal(sss.u32(dist), oracle.dist(ss, want, wl)), tag
        if p > 1 and not flags & sss.SSS_FLAG_MS:
            wa = oracle.doubling(ss, 0, oracle.default_kmax(ss), hseed)
            assert np.array_equal(sss.u32(approx), wa), tag + ("approx",)
        if len(strs) > 0 and rnd.random() < 0.2:
            hp, hl = _host_sort(sss, ss, p, prm)
            assert np.array_equal(hp, want), tag + ("host",)
            assert np.array_equal(hl, wl), tag + ("host",)
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
