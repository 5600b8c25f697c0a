"""Request loop for sorting requests on one GPU: HBM-budget admission and
continuous batching.

Every request is an independent string set to be sorted (permutation and LCP
array, ties by input index).  The server owns one device arena of exactly the
budget; every byte a request needs on the device (its characters, its string
table, its outputs and its share of the sorter's work memory) is a range of that
arena, so admission by arena allocation can never exceed the budget.

Scheduling (continuous batching): ``slots`` worker threads, each with its own
CUDA stream and sorter context.  Whenever a slot is free it takes the longest
FIFO prefix of the waiting requests whose memory it can allocate (within the
batch limits), generates or places their inputs, and sorts them all with one
sss_sort_batch call (each request is one instance of the batch).  Requests that
arrive while other batches run join the next batch of the next free slot; the
batches of different slots overlap on the device.  A batch's result for a
request does not depend on the other requests in it: the instances are
independent segments of one sort.

The scheduling and memory logic (RangeAllocator, Scheduler) is plain host code;
the device work is done by an engine (DeviceEngine here), so the host logic can
be exercised without a GPU.
"""
from __future__ import annotations

import bisect
import threading
import time
from dataclasses import dataclass, field

ALIGN = 256


def _align(x: int, a: int = ALIGN) -> int:
    return (x + a - 1) // a * a


class RangeAllocator:
    """First-fit allocator of byte ranges of a fixed-size arena (host side).

    Free ranges are kept sorted by offset and coalesced on free.  Every offset and
    size is a multiple of ``align``.  Not thread-safe by itself."""

    def __init__(self, size: int, align: int = ALIGN):
        self.align = align
        self.size = size // align * align
        self._free_off = [0] if self.size else []
        self._free_len = [self.size] if self.size else []
        self._live: dict[int, int] = {}
        self.used = 0
        self.high_water = 0

    def alloc(self, nbytes: int) -> int | None:
        n = max(self.align, _align(nbytes, self.align))
        for k, ln in enumerate(self._free_len):
            if ln >= n:
                off = self._free_off[k]
                if ln == n:
                    del self._free_off[k]
                    del self._free_len[k]
                else:
                    self._free_off[k] = off + n
                    self._free_len[k] = ln - n
                self._live[off] = n
                self.used += n
                self.high_water = max(self.high_water, self.used)
                return off
        return None

    def free(self, off: int) -> None:
        n = self._live.pop(off)
        self.used -= n
        k = bisect.bisect_left(self._free_off, off)
        # merge with the following free range
        if k < len(self._free_off) and off + n == self._free_off[k]:
            n += self._free_len[k]
            del self._free_off[k]
            del self._free_len[k]
        # merge with the preceding free range
        if k > 0 and self._free_off[k - 1] + self._free_len[k - 1] == off:
            self._free_len[k - 1] += n
        else:
            self._free_off.insert(k, off)
            self._free_len.insert(k, n)

    def largest_free(self) -> int:
        return max(self._free_len, default=0)

    def free_ranges(self) -> list[tuple[int, int]]:
        return list(zip(self._free_off, self._free_len))


@dataclass
class Request:
    """One sort request.  ``n`` strings of ``chars`` characters in total; the
    input is produced by the engine from (seed, n, ratio) or taken from
    ``payload`` (engine-specific).  Times are perf_counter seconds."""

    rid: int
    n: int
    chars: int
    seed: int = 0
    ratio: float = 0.5
    payload: object = None
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    state: str = "new"  # new, queued, running, done, error, rejected, cancelled
    error: str = ""
    slot: int = -1
    batch: int = -1
    perm: object = None
    lcp: object = None
    _chars_off: int = -1
    _group: object = None
    _event: threading.Event = field(default_factory=threading.Event)

    def wait(self, timeout: float | None = None) -> bool:
        """Block until the request has finished (done, error, rejected or
        cancelled) and the server's completion callback has run."""
        return self._event.wait(timeout)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class Batch:
    bid: int
    reqs: list
    first: list          # instance k = table strings first[k] .. first[k] + reqs[k].n - 1
    n_table: int
    keep_off: int        # arena range: string table and outputs (lives until every request is released)
    temp_off: int        # arena range: generator scratch and sorter work memory (freed at batch end)
    temp_bytes: int
    live: int = 0        # requests of the batch not yet released
    gen_ms: float = 0.0  # device time placing or generating the inputs
    sort_ms: float = 0.0  # device time of the sort


def batch_layout(n_table: int, sizes: list[int]):
    """Byte layout of a batch's kept range: offs u64, lens u32, perm u32, lcp u32
    (each 256-aligned).  Returns (offsets dict, total bytes)."""
    lay, off = {}, 0
    for name, w in (("offs", 8), ("lens", 4), ("perm", 4), ("lcp", 4)):
        lay[name] = off
        off += _align(w * max(1, n_table))
    return lay, off


class Scheduler:
    """Admission and batch formation (host logic only).

    batch_temp(n, m) gives the arena bytes of the transient work memory of a
    batch of m requests holding n strings in all.  The scheduler forms batches
    as FIFO prefixes of the queue that fit both the batch limits and the arena,
    and frees memory when batches end and requests are released.  The string
    limit bounds joining: a request larger than it runs in a batch of its own."""

    def __init__(self, arena_bytes: int, batch_temp, max_batch_requests: int = 256,
                 max_batch_strings: int = 1 << 24):
        self.alloc = RangeAllocator(arena_bytes)
        self.batch_temp = batch_temp
        self.max_req = max(1, max_batch_requests)
        self.max_strings = max(1, max_batch_strings)
        self.cv = threading.Condition()
        self.queue: list[Request] = []
        self.closed = False
        self.n_batches = 0
        self.inflight = 0
        self.batch_sizes: list[int] = []
        self.gen_ms = 0.0
        self.sort_ms = 0.0

    # -- request side ---------------------------------------------------------
    def min_bytes(self, req: Request) -> int:
        """Arena bytes a batch holding only this request needs."""
        return (_align(max(1, req.chars)) + batch_layout(req.n, [req.n])[1] + _align(self.batch_temp(req.n, 1)))

    def submit(self, req: Request) -> bool:
        with self.cv:
            if self.closed:
                raise RuntimeError("scheduler is closed")
            if req.n <= 0 or req.n >= (1 << 32):
                req.state, req.error = "rejected", "request size out of range"
            elif self.min_bytes(req) > self.alloc.size:
                req.state, req.error = "rejected", (f"request needs {self.min_bytes(req)} bytes, more than the "
                                                    f"{self.alloc.size}-byte budget")
            else:
                req.state = "queued"
                self.queue.append(req)
                self.cv.notify_all()
                return True
        req._event.set()
        return False

    def cancel(self, req: Request) -> bool:
        """Cancel a request that has not been admitted yet."""
        with self.cv:
            if req.state != "queued":
                return False
            self.queue.remove(req)
            req.state = "cancelled"
        req._event.set()
        return True

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()

    # -- slot side ------------------------------------------------------------
    def _try_take(self) -> Batch | None:
        reqs, offs, n_b = [], [], 0
        for req in self.queue:
            if len(reqs) == self.max_req or (reqs and n_b + req.n > self.max_strings):
                break
            off = self.alloc.alloc(max(1, req.chars))
            if off is None:
                break
            reqs.append(req)
            offs.append(off)
            n_b += req.n
        while reqs:
            sizes = [r.n for r in reqs]
            keep = self.alloc.alloc(batch_layout(n_b, sizes)[1])
            tb = self.batch_temp(n_b, len(reqs))
            temp = self.alloc.alloc(tb) if keep is not None else None
            if keep is not None and temp is not None:
                break
            if keep is not None:
                self.alloc.free(keep)
            last = reqs.pop()
            self.alloc.free(offs.pop())
            n_b -= last.n
        if not reqs:
            return None
        first, f = [], 0
        for r, o in zip(reqs, offs):
            r._chars_off = o
            first.append(f)
            f += r.n
        del self.queue[:len(reqs)]
        b = Batch(self.n_batches, reqs, first, n_b, keep, temp, tb, live=len(reqs))
        self.n_batches += 1
        self.inflight += 1
        self.batch_sizes.append(len(reqs))
        now = time.perf_counter()
        for r in reqs:
            r.state, r.t_admit, r._group, r.batch = "running", now, b, b.bid
        return b

    def next_batch(self) -> Batch | None:
        """Block until a batch can be formed (None once closed and drained)."""
        with self.cv:
            while True:
                if self.queue:
                    b = self._try_take()
                    if b is not None:
                        return b
                elif self.closed:
                    return None
                self.cv.wait(0.05)

    def batch_done(self, b: Batch, error: str = ""):
        now = time.perf_counter()
        with self.cv:
            self.alloc.free(b.temp_off)
            self.inflight -= 1
            self.gen_ms += b.gen_ms
            self.sort_ms += b.sort_ms
            for r in b.reqs:
                r.t_done = now
                if error:
                    r.state, r.error = "error", error
                elif r.state == "running":
                    r.state = "done"
            self.cv.notify_all()

    def release(self, req: Request):
        """Give a finished request's device memory back to the arena."""
        with self.cv:
            b = req._group
            if b is None:
                return
            req._group = None
            req.perm = req.lcp = None
            self.alloc.free(req._chars_off)
            req._chars_off = -1
            b.live -= 1
            if b.live == 0:
                self.alloc.free(b.keep_off)
            self.cv.notify_all()


class DeviceEngine:
    """Device side of the server: a budget-sized arena, one stream and sorter
    context per slot, request inputs generated on the device, batches sorted by
    sss_sort_batch with the context's work memory taken from the arena."""

    def __init__(self, device: int, budget_bytes: int, prm=None):
        import torch

        from . import params
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.arena = torch.empty(budget_bytes, dtype=torch.uint8, device=self.device)
        self.prm = prm or params()

    @staticmethod
    def gen_bytes(n_table: int, m: int) -> int:
        """Bound on the generator's scratch for a batch: the request descriptors
        (64 bytes each), then one u64 per 4096 strings of each request, rounded
        up per request to whole 256-byte ranges."""
        return _align(64 * m) + _align(8 * (n_table // 4096) + m * (8 + ALIGN) + ALIGN)

    def batch_temp(self, n_table: int, m: int) -> int:
        from . import batch_workspace_bytes
        return self.gen_bytes(n_table, m) + _align(batch_workspace_bytes(n_table, m, self.prm))

    def make_slot(self, i: int):
        from . import Context
        torch = self.torch
        st = torch.cuda.Stream(self.device)
        with torch.cuda.stream(st):
            ctx = Context(self.device.index)
        return {"stream": st, "ctx": ctx}

    def _view(self, off: int, count: int, dtype):
        torch = self.torch
        w = torch.empty((), dtype=dtype).element_size()
        return self.arena[off: off + w * max(1, count)].view(dtype)

    def run(self, slot, b: Batch):
        torch = self.torch
        st, ctx = slot["stream"], slot["ctx"]
        lay, _ = batch_layout(b.n_table, [r.n for r in b.reqs])
        offs = self._view(b.keep_off + lay["offs"], b.n_table, torch.int64)
        lens = self._view(b.keep_off + lay["lens"], b.n_table, torch.int32)
        perm = self._view(b.keep_off + lay["perm"], b.n_table, torch.int32)
        lcp = self._view(b.keep_off + lay["lcp"], b.n_table, torch.int32)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        m = len(b.reqs)
        try:
            self._run_on_stream(st, ctx, b, lay, offs, lens, perm, lcp, ev, m)
        finally:
            # whatever happened, the arena ranges of this batch go back to the
            # allocator only once no kernel of it can still touch them
            st.synchronize()
            ctx.set_workspace(None)
        b.gen_ms = ev[0].elapsed_time(ev[1])
        b.sort_ms = ev[1].elapsed_time(ev[2])
        for r, f in zip(b.reqs, b.first):
            r.perm, r.lcp = perm[f:f + r.n], lcp[f:f + r.n]

    def _run_on_stream(self, st, ctx, b: Batch, lay, offs, lens, perm, lcp, ev, m: int):
        torch = self.torch
        import datagen.cuda as dgc

        from . import sss_sort_batch
        with torch.cuda.stream(st):
            ev[0].record(st)
            gen_off = b.temp_off + _align(64 * m)
            if all(r.payload is None for r in b.reqs):
                # every request generated on the device in one launch sequence
                desc = dgc.request_descs([r.seed for r in b.reqs], [r.n for r in b.reqs], [r.ratio for r in b.reqs],
                                         [r._chars_off for r in b.reqs])
                d_desc = self.arena[b.temp_off: b.temp_off + desc.nbytes]
                d_desc.copy_(torch.from_numpy(desc.view("uint8")))
                words = dgc.request_scratch_words(b.n_table) + m
                dgc.request_batch_into(self.arena, offs, lens, perm, self._view(gen_off, words, torch.int64), d_desc,
                                       m, b.n_table)
            else:
                for r, f in zip(b.reqs, b.first):
                    words = dgc.request_scratch_words(r.n)
                    if r.payload is not None:
                        self._place(r, f, offs, lens)
                    else:
                        dgc.request_into(self.arena, r._chars_off, offs[f:f + r.n], lens[f:f + r.n],
                                         perm[f:f + r.n], self._view(gen_off, words, torch.int64), r.seed, r.n,
                                         r.ratio)
                    gen_off += _align(8 * words)
            ev[1].record(st)
            ws_off = b.temp_off + self.gen_bytes(b.n_table, len(b.reqs))
            ctx.set_workspace(self.arena[ws_off: ws_off + self._ws(b)])
            sss_sort_batch(self.arena, offs[:b.n_table], lens[:b.n_table], b.first, [r.n for r in b.reqs], self.prm,
                           out_perm=perm[:b.n_table], out_lcp=lcp[:b.n_table], ctx=ctx)
            ev[2].record(st)

    def _ws(self, b: Batch) -> int:
        from . import batch_workspace_bytes
        return batch_workspace_bytes(b.n_table, len(b.reqs), self.prm)

    def _place(self, r: Request, f: int, offs, lens):
        """Copy a request given as host (chars u8, lens i32) arrays into the arena."""
        torch = self.torch
        h_chars, h_lens = r.payload
        h_chars = torch.as_tensor(h_chars)
        h_lens = torch.as_tensor(h_lens)
        self.arena[r._chars_off: r._chars_off + h_chars.numel()].copy_(h_chars, non_blocking=True)
        l64 = h_lens.to(torch.int64)
        o = torch.cumsum(l64, 0) - l64 + r._chars_off
        offs[f:f + r.n].copy_(o, non_blocking=True)
        lens[f:f + r.n].copy_(h_lens, non_blocking=True)

    def close(self):
        self.arena = None


class Server:
    """Sorting server on one GPU (see the module docstring)."""

    def __init__(self, device: int = 0, budget_bytes: int = 64 << 30, slots: int = 4, max_batch_requests: int = 256,
                 max_batch_strings: int = 1 << 24, prm=None, engine=None, keep_results: bool = False,
                 on_done=None):
        self.engine = engine if engine is not None else DeviceEngine(device, budget_bytes, prm)
        self.sched = Scheduler(budget_bytes, self.engine.batch_temp, max_batch_requests, max_batch_strings)
        self.keep = keep_results
        self.on_done = on_done
        self.done: list[Request] = []
        self._lock = threading.Lock()
        self._slots = [self.engine.make_slot(i) for i in range(slots)]
        self._threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        for t in self._threads:
            t.start()

    def _worker(self, i: int):
        slot = self._slots[i]
        while True:
            b = self.sched.next_batch()
            if b is None:
                return
            for r in b.reqs:
                r.slot = i
            err = ""
            try:
                self.engine.run(slot, b)
            except Exception as ex:  # the batch fails; the server keeps serving
                err = f"{type(ex).__name__}: {ex}"
            self.sched.batch_done(b, err)
            for r in b.reqs:
                with self._lock:
                    self.done.append(r)
                if self.on_done is not None:
                    try:
                        self.on_done(r)
                    except Exception as ex:  # a failing callback must not stop the slot
                        r.error = r.error or f"on_done: {type(ex).__name__}: {ex}"
                if not self.keep or r.state != "done":
                    self.sched.release(r)
                r._event.set()

    def submit(self, req: Request) -> bool:
        if not req.t_arrival:
            req.t_arrival = time.perf_counter()
        ok = self.sched.submit(req)
        if not ok:
            with self._lock:
                self.done.append(req)
        return ok

    def cancel(self, req: Request) -> bool:
        ok = self.sched.cancel(req)
        if ok:
            with self._lock:
                self.done.append(req)
        return ok

    def release(self, req: Request):
        self.sched.release(req)

    def close(self):
        self.sched.close()
        for t in self._threads:
            t.join()
        if hasattr(self.engine, "close"):
            self.engine.close()

    def run_open_loop(self, reqs: list[Request], arrival_s: list[float]) -> float:
        """Submit reqs[k] at arrival_s[k] seconds after now (latency counts from
        the scheduled arrival), wait for all; returns the start time."""
        t0 = time.perf_counter()
        for r, a in zip(reqs, arrival_s):
            t = t0 + a
            d = t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            r.t_arrival = t
            self.submit(r)
        for r in reqs:
            r.wait()
        return t0

    def run_closed_loop(self, reqs: list[Request]) -> float:
        """Submit everything at once (saturation); returns the start time."""
        t0 = time.perf_counter()
        for r in reqs:
            r.t_arrival = t0
            self.submit(r)
        for r in reqs:
            r.wait()
        return t0


def summarize(reqs: list[Request], t0: float) -> dict:
    """Latency percentiles and throughput of finished requests."""
    ok = [r for r in reqs if r.state == "done"]
    if not ok:
        return {"requests": len(reqs), "done": 0}
    lat = sorted(r.latency for r in ok)
    svc = sorted(r.t_done - r.t_admit for r in ok)

    def pct(a, q):
        return a[min(len(a) - 1, max(0, int(round(q * (len(a) - 1)))))]

    span = max(r.t_done for r in ok) - t0
    chars = sum(r.chars for r in ok)
    strings = sum(r.n for r in ok)
    return {"requests": len(reqs), "done": len(ok),
            "errors": sum(r.state == "error" for r in reqs),
            "rejected": sum(r.state == "rejected" for r in reqs),
            "p50_ms": 1e3 * pct(lat, 0.50), "p99_ms": 1e3 * pct(lat, 0.99), "mean_ms": 1e3 * sum(lat) / len(lat),
            "service_p50_ms": 1e3 * pct(svc, 0.50), "service_p99_ms": 1e3 * pct(svc, 0.99),
            "chars_per_s": chars / span, "strings_per_s": strings / span, "requests_per_s": len(ok) / span,
            "chars": chars, "strings": strings, "span_s": span}
