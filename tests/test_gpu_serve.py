"""Request loop on the GPU: every request's result in the mix (continuous
batching, several slots, a tight budget) equals its result alone, bit-exact;
small requests equal the oracle; admission stays within the budget; failures,
rejections and cancellations are reported without disturbing other requests."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(count, seed, cap):
    import datagen.cuda as dgc
    from paper_2404_16517_gb300.serve import Request
    sizes, ratios, _, seeds = datagen.config5_requests(count, seed=seed)
    sizes = np.minimum(sizes, cap)
    sizes[:4] = [1, 2, 3, 4097][:4]  # edge sizes: one string, tiny, just past a scan chunk
    tot = dgc.request_totals(seeds, sizes)
    return [Request(rid=i, n=int(sizes[i]), chars=int(tot[i]), seed=int(seeds[i]), ratio=float(ratios[i]))
            for i in range(count)]


def _serve(reqs, **kw):
    from paper_2404_16517_gb300.serve import Server
    got = {}

    def grab(r):
        if r.state == "done":
            got[r.rid] = (r.perm.cpu().numpy().view(np.uint32).copy(), r.lcp.cpu().numpy().view(np.uint32).copy())
    srv = Server(on_done=grab, **kw)
    srv.run_closed_loop(reqs)
    hw = srv.sched.alloc.high_water
    used = srv.sched.alloc.used
    srv.close()
    return got, hw, used


def test_mix_equals_alone_and_oracle():
    reqs = _requests(48, seed=11, cap=30000)
    budget = 96 << 20
    mix, hw, used = _serve(_fresh(reqs), budget_bytes=budget, slots=4,
                           max_batch_requests=16)
    assert hw <= budget and used == 0
    alone, _, _ = _serve(_fresh(reqs), budget_bytes=budget, slots=1, max_batch_requests=1)
    assert sorted(mix) == sorted(alone) == list(range(48))
    for i in range(48):
        assert np.array_equal(mix[i][0], alone[i][0]), f"request {i} perm"
        assert np.array_equal(mix[i][1], alone[i][1]), f"request {i} lcp"
    # small requests against the oracle, on the same generated characters
    for r in reqs:
        if r.n > 3000:
            continue
        ss = _request_strings(r)
        want = oracle.sort(ss)
        assert np.array_equal(mix[r.rid][0], want), f"request {r.rid} vs oracle"
        assert np.array_equal(mix[r.rid][1], oracle.lcp_array(ss, want))


def _fresh(reqs):
    from paper_2404_16517_gb300.serve import Request
    return [Request(rid=r.rid, n=r.n, chars=r.chars, seed=r.seed, ratio=r.ratio) for r in reqs]


def _request_strings(r):
    import datagen.cuda as dgc
    chars = torch.zeros(max(1, r.chars), dtype=torch.uint8, device="cuda")
    offs = torch.empty(r.n, dtype=torch.int64, device="cuda")
    lens = torch.empty(r.n, dtype=torch.int32, device="cuda")
    cp = torch.empty(r.n, dtype=torch.int32, device="cuda")
    sc = torch.empty(dgc.request_scratch_words(r.n), dtype=torch.int64, device="cuda")
    dgc.request_into(chars, 0, offs, lens, cp, sc, r.seed, r.n, r.ratio)
    torch.cuda.synchronize()
    return datagen.StringSet(chars.cpu().numpy(), offs.cpu().numpy().view(np.uint64),
                             lens.cpu().numpy().view(np.uint32))


def test_request_generator_totals_and_placement():
    import datagen.cuda as dgc
    reqs = _requests(6, seed=13, cap=20000)
    for r in reqs:
        assert r.chars == datagen.request_chars(r.seed, r.n)
        ss = _request_strings(r)
        assert int(ss.lens.astype(np.int64).sum()) == r.chars
        assert ss.lens.min() >= 16 and ss.lens.max() <= 1000
        # the same request placed at another offset has the same characters
        base = 4096 + 37
        chars = torch.zeros(base + r.chars, dtype=torch.uint8, device="cuda")
        offs = torch.empty(r.n, dtype=torch.int64, device="cuda")
        lens = torch.empty(r.n, dtype=torch.int32, device="cuda")
        cp = torch.empty(r.n, dtype=torch.int32, device="cuda")
        sc = torch.empty(dgc.request_scratch_words(r.n), dtype=torch.int64, device="cuda")
        dgc.request_into(chars, base, offs, lens, cp, sc, r.seed, r.n, r.ratio)
        torch.cuda.synchronize()
        o = offs.cpu().numpy()
        assert o[0] == base
        assert np.array_equal(o - base, ss.offs.astype(np.int64))
        assert np.array_equal(chars[base:].cpu().numpy(), ss.chars[:r.chars])


def test_budget_pressure_open_loop():
    from paper_2404_16517_gb300.serve import Server, summarize
    reqs = _fresh(_requests(40, seed=17, cap=60000))
    budget = 64 << 20
    srv = Server(budget_bytes=budget, slots=3, max_batch_requests=8)
    t0 = srv.run_open_loop(reqs, [0.0005 * k for k in range(len(reqs))])
    srv.close()
    st = summarize(reqs, t0)
    fits = [r for r in reqs if srv.sched.min_bytes(r) <= budget]
    assert st["done"] == len(fits)
    assert all(r.state == "rejected" for r in reqs if r not in fits)
    assert srv.sched.alloc.high_water <= budget and srv.sched.alloc.used == 0


def test_failed_batch_does_not_disturb_others():
    import paper_2404_16517_gb300 as sss
    from paper_2404_16517_gb300.serve import DeviceEngine, Server

    class Faulty(DeviceEngine):
        def run(self, slot, b):
            if any(r.rid == 3 for r in b.reqs):
                # a bad argument: an instance with p = 2 is refused on the host
                arr = (sss.sss_instance * 1)()
                arr[0].first, arr[0].n, arr[0].p = 0, 1, 2
                z = self.arena[:1]
                st = sss.lib().sss_sort_batch(slot["ctx"].h, z.data_ptr(), 1, z.data_ptr(), z.data_ptr(), 1, arr, 1,
                                              None, z.data_ptr(), z.data_ptr(), None)
                slot["ctx"]._check(st, slot["ctx"].h)
            return super().run(slot, b)

    reqs = _fresh(_requests(8, seed=19, cap=5000))
    eng = Faulty(0, 64 << 20)
    srv = Server(budget_bytes=64 << 20, slots=2, max_batch_requests=1, engine=eng, keep_results=True)
    srv.run_closed_loop(reqs)
    assert reqs[3].state == "error" and "p > 1" in reqs[3].error
    for r in reqs:
        if r.rid != 3:
            assert r.state == "done"
            ss = _request_strings(r)
            want = oracle.sort(ss)
            assert np.array_equal(r.perm.cpu().numpy().view(np.uint32), want)
            srv.release(r)
    srv.close()
    assert srv.sched.alloc.used == 0


def test_batched_generator_equals_single_requests():
    import datagen.cuda as dgc
    reqs = _requests(9, seed=23, cap=9000)
    gap = 1000  # characters left unused between requests
    bases, b = [], 64
    for r in reqs:
        bases.append(b)
        b += r.chars + gap
    chars = torch.zeros(b, dtype=torch.uint8, device="cuda")
    n = sum(r.n for r in reqs)
    offs = torch.empty(n, dtype=torch.int64, device="cuda")
    lens = torch.empty(n, dtype=torch.int32, device="cuda")
    cp = torch.empty(n, dtype=torch.int32, device="cuda")
    sc = torch.empty(dgc.request_scratch_words(n) + len(reqs), dtype=torch.int64, device="cuda")
    desc = dgc.request_descs([r.seed for r in reqs], [r.n for r in reqs], [r.ratio for r in reqs], bases)
    d_desc = torch.from_numpy(desc.view(np.uint8)).cuda()
    dgc.request_batch_into(chars, offs, lens, cp, sc, d_desc, len(reqs), n)
    torch.cuda.synchronize()
    C, O, L = chars.cpu().numpy(), offs.cpu().numpy(), lens.cpu().numpy()
    f = 0
    for r, base in zip(reqs, bases):
        ss = _request_strings(r)
        assert np.array_equal(L[f:f + r.n], ss.lens.view(np.int32))
        assert np.array_equal(O[f:f + r.n] - base, ss.offs.astype(np.int64))
        assert np.array_equal(C[base:base + r.chars], ss.chars[:r.chars])
        f += r.n
