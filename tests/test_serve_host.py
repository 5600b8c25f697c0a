"""Host logic of the request loop (no GPU): the arena range allocator, budget
admission, FIFO batch formation, cancellation, rejection and failure handling,
with a fake engine that sleeps instead of sorting."""
import random
import threading
import time

import pytest

from paper_2404_16517_gb300.serve import ALIGN, RangeAllocator, Request, Scheduler, Server, summarize


def _check_allocator(a: RangeAllocator, live: dict):
    # live ranges disjoint and inside the arena; free list sorted, coalesced and
    # complementary to the live ranges
    spans = sorted((o, n) for o, n in live.items())
    for (o1, n1), (o2, _) in zip(spans, spans[1:]):
        assert o1 + n1 <= o2
    for o, n in spans:
        assert 0 <= o and o + n <= a.size and o % ALIGN == 0 and n % ALIGN == 0
    fr = a.free_ranges()
    for (o1, n1), (o2, _) in zip(fr, fr[1:]):
        assert o1 + n1 < o2, "adjacent free ranges not coalesced"
    assert sum(n for _, n in fr) + sum(n for _, n in spans) == a.size
    assert a.used == sum(n for _, n in spans)
    covered = sorted(spans + fr)
    pos = 0
    for o, n in covered:
        assert o == pos
        pos += n
    assert pos == a.size


def test_allocator_random():
    rnd = random.Random(7)
    a = RangeAllocator(1 << 20)
    live = {}
    for step in range(4000):
        if live and (rnd.random() < 0.45 or a.largest_free() < ALIGN):
            off = rnd.choice(list(live))
            a.free(off)
            del live[off]
        else:
            want = rnd.choice([1, 100, 256, 257, 5000, 40000, 1 << 17])
            off = a.alloc(want)
            if off is None:
                # first fit fails only when no free range is large enough
                assert a.largest_free() < (want + ALIGN - 1) // ALIGN * ALIGN
            else:
                live[off] = max(ALIGN, (want + ALIGN - 1) // ALIGN * ALIGN)
        if step % 50 == 0:
            _check_allocator(a, live)
    for off in list(live):
        a.free(off)
    assert a.used == 0 and a.free_ranges() == [(0, a.size)]


class FakeEngine:
    """Sleeps in proportion to the batch size; fails batches holding a request
    whose seed is marked bad; records every batch."""

    def __init__(self, bad_seeds=()):
        self.bad = set(bad_seeds)
        self.batches = []
        self.lock = threading.Lock()
        self.overlap = 0
        self.active = 0

    def batch_temp(self, n, m):
        return 64 * n + 512 * m

    def make_slot(self, i):
        return {"i": i}

    def run(self, slot, b):
        with self.lock:
            self.batches.append([r.rid for r in b.reqs])
            self.active += 1
            self.overlap = max(self.overlap, self.active)
        try:
            time.sleep(0.002 + 1e-7 * b.n_table)
            if any(r.seed in self.bad for r in b.reqs):
                raise RuntimeError("injected failure: bad argument")
            for r in b.reqs:
                r.perm = ("perm", r.rid)
        finally:
            with self.lock:
                self.active -= 1


def _reqs(count, seed=3, max_n=4000):
    rnd = random.Random(seed)
    out = []
    for i in range(count):
        n = rnd.randint(1, max_n)
        out.append(Request(rid=i, n=n, chars=n * rnd.randint(16, 1000), seed=i))
    return out


@pytest.mark.parametrize("slots", [1, 3])
def test_budget_fifo_and_release(slots):
    budget = 24 << 20
    eng = FakeEngine()
    seen = []
    srv = Server(budget_bytes=budget, slots=slots, engine=eng, max_batch_requests=8,
                 on_done=lambda r: seen.append((r.rid, r.perm)))
    reqs = _reqs(120)
    t0 = srv.run_closed_loop(reqs)
    srv.close()
    assert all(r.state == "done" for r in reqs)
    assert sorted(rid for rid, _ in seen) == list(range(120))
    assert all(p == ("perm", rid) for rid, p in seen)
    # admission within the budget, everything released at the end
    assert srv.sched.alloc.high_water <= budget
    assert srv.sched.alloc.used == 0
    # batches are FIFO prefixes: admission order is submission order
    order = [rid for b in eng.batches for rid in b]
    assert order == list(range(120))
    assert max(len(b) for b in eng.batches) <= 8
    if slots > 1:
        assert eng.overlap > 1, "batches of different slots should overlap"
    s = summarize(reqs, t0)
    assert s["done"] == 120 and s["p99_ms"] >= s["p50_ms"] > 0


def test_continuous_batching_joins_waiting_requests():
    # one slot busy with a long batch: requests arriving meanwhile form the next batch together
    eng = FakeEngine()
    srv = Server(budget_bytes=64 << 20, slots=1, engine=eng, max_batch_requests=64)
    first = Request(rid=0, n=200000, chars=1 << 20)
    srv.submit(first)
    time.sleep(0.005)
    later = [Request(rid=k, n=100, chars=2000) for k in range(1, 6)]
    for r in later:
        srv.submit(r)
    for r in [first] + later:
        assert r.wait(10)
    srv.close()
    assert eng.batches[0] == [0]
    assert eng.batches[1] == [1, 2, 3, 4, 5]


def test_reject_cancel_and_failure():
    eng = FakeEngine(bad_seeds={5})
    srv = Server(budget_bytes=8 << 20, slots=2, engine=eng, max_batch_requests=1)
    big = Request(rid=100, n=10, chars=9 << 20, seed=100)       # larger than the whole budget
    assert not srv.submit(big)
    assert big.state == "rejected" and "budget" in big.error
    # fill the queue behind a slow request, then cancel one that is still queued
    blockers = [Request(rid=k, n=2000, chars=1 << 20, seed=k) for k in range(6)]
    for r in blockers:
        srv.submit(r)
    late = Request(rid=50, n=10, chars=100, seed=50)
    srv.submit(late)
    cancelled = srv.cancel(late)
    for r in blockers:
        assert r.wait(10)
    srv.close()
    if cancelled:
        assert late.state == "cancelled"
    assert blockers[5].state == "error" and "injected" in blockers[5].error
    assert all(r.state == "done" for r in blockers[:5])
    assert srv.sched.alloc.used == 0


def test_open_loop_latency_accounting():
    eng = FakeEngine()
    srv = Server(budget_bytes=32 << 20, slots=2, engine=eng)
    reqs = _reqs(40, seed=9, max_n=500)
    arrivals = [0.001 * k for k in range(40)]
    t0 = srv.run_open_loop(reqs, arrivals)
    srv.close()
    for r, a in zip(reqs, arrivals):
        assert r.t_arrival == pytest.approx(t0 + a, abs=1e-9)
        assert r.t_done >= r.t_admit >= r.t_arrival
    s = summarize(reqs, t0)
    assert s["done"] == 40 and s["chars"] == sum(r.chars for r in reqs)


def test_batches_respect_the_string_limit():
    # requests join a batch only while the batch's string count stays within the
    # limit; a request larger than the limit still runs, in a batch of its own
    eng = FakeEngine()
    srv = Server(budget_bytes=256 << 20, slots=1, engine=eng, max_batch_requests=64, max_batch_strings=1000)
    blocker = Request(rid=0, n=50000, chars=1 << 20)  # holds the slot while the rest queue up
    srv.submit(blocker)
    time.sleep(0.005)
    sizes = [400, 400, 400, 1500, 300, 300, 300, 300]
    reqs = [Request(rid=k + 1, n=n, chars=10 * n) for k, n in enumerate(sizes)]
    for r in reqs:
        srv.submit(r)
    for r in [blocker] + reqs:
        assert r.wait(10)
    srv.close()
    by_rid = {r.rid: r.n for r in [blocker] + reqs}
    batches = eng.batches[1:]
    assert [rid for b in batches for rid in b] == list(range(1, len(sizes) + 1))  # FIFO
    for b in batches:
        total = sum(by_rid[rid] for rid in b)
        assert total <= 1000 or len(b) == 1, (b, total)
    assert [4] in batches  # the 1500-string request alone
