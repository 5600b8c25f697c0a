#!/usr/bin/env python
"""Benchmark of the string sorter on one or more GB300s (one replica per GPU).

Workload (default): the full prefix-doubling merge sort of 4,194,304 strings of
500 characters over A-Z in p = 16 partitions (chars 0-241 from one of 64
seeded templates, the rest uniform; D/N about 0.5), generated on the device.
A step is one sss_sort call over the whole set (local sort, prefix doubling,
partition, LCP-compressed exchange, LCP merge, plus dist).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank sorts its own copy of
the workload (replicas, weak scaling); value = all ranks' characters / the
slowest rank's time.  ``--impl reference`` times the plain-C oracle on a
bounded sample of the same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sorted chars/s and strings/s on 1 GB300 (% of HBM roofline); p50/p99 request latency"
WORKLOAD = "pdms_4194304x500_AZ_T64_shared242_p16"
N_FULL, LEN, P = 4194304, 500, 16
CPU_SAMPLE = 1 << 17  # strings of the CPU-baseline sample (both oracle modes)
REF_SAMPLE = 1 << 19  # strings per step of the reference arm (all host cores)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def lib_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2404_16517_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, ws: int) -> float:
    """Largest value of x over all ranks (x itself at world size 1).  NCCL
    reduces a device tensor; gloo a host tensor."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, seconds_max: float) -> float:
    """Whole-job throughput of ws replicas: all ranks' units over the slowest
    rank's time."""
    return units_per_rank * ws / seconds_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the report."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_sample(n: int):
    """The first n strings of the full-pipeline workload, from the same
    generator the GPU run uses (device generator when a GPU is present)."""
    import numpy as np

    import datagen
    try:
        import torch
        import datagen.cuda as dgc
        if torch.cuda.is_available():
            c, o, l = dgc.config2(N_FULL, 0, n)
            return datagen.StringSet(c.cpu().numpy(), o.cpu().numpy().view(np.uint64),
                                     l.cpu().numpy().view(np.uint32))
    except Exception:
        pass
    return datagen.config2(N_FULL, 0, n)


def _time_runs(fn, runs: int, warm: int = 1):
    """The paper's timing rule: `warm` untimed runs, then the mean of `runs` runs."""
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return statistics.mean(ts), ts


def cpu_baseline(n: int, runs: int = 5):
    """The oracle pipeline (p = 16, v = 2, k = 0..9) on the host cores, two
    modes on the same sample: one thread (the definition) and every core
    (partitions, key ranges and buckets shared out among threads; the reported
    baseline).  Each is one warm-up run, then the mean of `runs` runs."""
    import oracle
    ss = _oracle_sample(n)
    cores = os.cpu_count() or 1
    t1, _ = _time_runs(lambda: oracle.pdms(ss, P, 2, 0, 9, 0), runs)
    tn, _ = _time_runs(lambda: oracle.pdms_parallel(ss, P, 2, 0, 9, 0, nthreads=cores), runs)
    chars = n * LEN
    return {"value": chars / tn, "unit": "chars/s", "cores": cores, "kind": "oracle",
            "strings_per_s": n / tn, "cpu_model": cpu_model(),
            "sample": f"first {n} of the {N_FULL} strings (same generator), p={P}, v=2, k=0..9; "
                      f"one warm-up then the mean of {runs} runs per mode",
            "single_thread": {"value": chars / t1, "unit": "chars/s", "cores": 1, "s_per_run": t1},
            "all_cores": {"value": chars / tn, "unit": "chars/s", "cores": cores, "s_per_run": tn}}


def run_reference(args, ws, rank):
    """The oracle pipeline on every host core, on a bounded sample of the
    workload (rank 0 only; other ranks exit without work)."""
    if rank != 0:
        return 0
    import oracle

    n = args.cpu_sample
    ss = _oracle_sample(n)
    cores = os.cpu_count() or 1
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.pdms_parallel(ss, P, 2, 0, 9, 0, nthreads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
        if s == 0 and args.steps + args.warmup > 1 and dt * (args.steps + args.warmup) > 240:
            # keep the whole reference run within a few minutes
            args.steps = max(1, int(240 // dt) - args.warmup)
    t = statistics.mean(times)
    chars = n * LEN
    value = chars / t
    sample = (f"first {n} of the {N_FULL} strings (same generator), p={P}; one oracle PDMS pass per step on "
              f"{cores} host threads; mean of the timed steps")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "chars/s", "n_gpus": ws,
           "steps": len(times), "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "strings_per_s": n / t,
           "config": {"workload": WORKLOAD, "sample_strings": n, "partitions": P},
           "cpu_baseline": {"value": value, "unit": "chars/s", "cores": cores, "kind": "oracle", "sample": sample,
                            "cpu_model": cpu_model()},
           "e2e": {"value": value, "unit": "chars/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help=f"oracle sample in strings (default {CPU_SAMPLE}; {REF_SAMPLE} for --impl reference)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--breakdown", action="store_true", help="per-kernel times to stderr")
    ap.add_argument("--merge-ms", type=int, default=0, help="merge segment spacing (0 = library default)")
    ap.add_argument("--p", type=int, default=P, help="partitions (profiling of smaller cases)")
    ap.add_argument("--workload", default="all",
                    choices=["all", "pdms", "batch", "serve", "charsample", "suffix", "config1", "config3", "h2d"])
    ap.add_argument("--batch-instances", type=int, default=4096)
    ap.add_argument("--no-tune", action="store_true", help="batch: skip the autotuner (default knobs)")
    ap.add_argument("--no-graph", action="store_true", help="batch: host-driven round loop only")
    ap.add_argument("--per-instance-steps", type=int, default=2,
                    help="timed passes of one sss_sort call per instance (0: skip that comparison)")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-warmup", type=int, default=1000)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-max-batch", type=int, default=256)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, local = dist_env()
    if args.cpu_sample is None:
        args.cpu_sample = REF_SAMPLE if args.impl == "reference" else CPU_SAMPLE
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import numpy as np
    import torch

    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as sss

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    if args.workload == "h2d":
        if rank == 0:
            print(json.dumps({"metric": "host link GB/s", "n_gpus": ws, **bench_h2d(args, dev)}), flush=True)
        return 0
    if args.workload in ("batch", "serve", "charsample", "suffix", "config1", "config3"):
        ctx = sss.context(local)
        res = {"batch": bench_batch, "charsample": bench_charsample, "suffix": bench_suffix,
               "config1": bench_config1, "config3": bench_config3}.get(args.workload, None)
        res = res(args, dev, ctx) if res else bench_serve(args, dev)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "n_gpus": ws, **res}), flush=True)
        return 0

    n = args.n
    chars, offs, lens = dgc.config2(n, 0, n)
    N = n * LEN
    ctx = sss.context(local)
    prm = sss.params(merge_ms=args.merge_ms)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    dist_t = torch.empty(n, dtype=torch.int32, device=dev)
    approx = torch.empty(n, dtype=torch.int32, device=dev)

    def step(prm_=None):
        sss.sss_sort(chars, offs, lens, args.p, prm_ or prm, perm, lcp, out_dist=dist_t, out_approx=approx, ctx=ctx)

    # the local sort's round loop host-driven or as one graph launch: the faster
    # is timed below (both are reported)
    def loop_ms(prm_, reps=5):
        for _ in range(2):
            step(prm_)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            step(prm_)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    prm_host = prm
    prm_graph = sss.params(merge_ms=args.merge_ms, flags=sss.SSS_FLAG_GRAPH)
    round_loop = {"ms_host_loop": loop_ms(prm_host), "ms_graph": loop_ms(prm_graph)}
    round_loop["used"] = "graph" if round_loop["ms_graph"] < round_loop["ms_host_loop"] else "host"
    if round_loop["used"] == "graph":
        prm = prm_graph

    # warm-up; the second one with every kernel timed (host-driven, so that the
    # kernels inside a graph launch are timed one by one) to find the dominant kernel
    step()
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_timing(True, "")
    step(prm_host)
    torch.cuda.synchronize()
    stats_all = ctx.kernel_stats()
    ctx.set_timing(False)
    for _ in range(args.warmup - 2):
        step()
    torch.cuda.synchronize()
    dom = max(stats_all.items(), key=lambda kv: kv[1]["total_ms"])[0]
    D = int(dist_t.to(torch.int64).sum().item())
    Dapprox = int(approx.to(torch.int64).sum().item())
    sum_lcp = int(lcp.to(torch.int64).sum().item())

    # timed region: events on the context stream, the dominant kernel timed too
    ctx.reset_stats()
    ctx.set_timing(True, dom)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    stats = ctx.kernel_stats()
    ctx.set_timing(False)
    launches = sum(v["launches"] for v in stats.values())
    ms = max_over_ranks(ms, ws)
    ms_step = ms / args.steps
    value = job_rate(N, ws, ms_step / 1e3)

    # roofline of the dominant kernel
    hbm, peak_kind = peaks()
    dstat = stats.get(dom, {"launches": 0, "total_ms": 0.0, "timed": 0})
    per_step = args.steps
    if dstat["timed"] == 0:  # the dominant kernel ran inside the graph: its host-driven time
        dstat, per_step = stats_all.get(dom), 1
    avg_ms = dstat["total_ms"] / max(1, dstat["timed"])
    algo = algorithmic_bytes(dom, n, N, D, Dapprox, dstat["launches"] / max(1, per_step))
    achieved = algo / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    traffic = known_traffic(dom)

    # end to end: host buffers, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        h_chars = torch.empty(chars.numel(), dtype=torch.uint8, pin_memory=True)
        h_chars.copy_(chars)
        h_offs = offs.cpu().pin_memory()
        h_lens = lens.cpu().pin_memory()
        h_perm = torch.empty(n, dtype=torch.int32, pin_memory=True)
        h_lcp = torch.empty(n, dtype=torch.int32, pin_memory=True)
        d_chars = torch.empty_like(chars)
        d_offs = torch.empty_like(offs)
        d_lens = torch.empty_like(lens)

        def e2e_step():
            # the public host-input call: views uploaded, then the characters one
            # partition chunk at a time while the partitions already in are
            # sorted; outputs copied back into pinned host memory
            sss.sss_sort_host(h_chars, h_offs, h_lens, args.p, d_chars, d_offs, d_lens, prm, perm, lcp, h_perm,
                              h_lcp, ctx=ctx)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(st)
        for _ in range(args.e2e_steps):
            e2e_step()
        a1.record(st)
        torch.cuda.synchronize()
        ems = max_over_ranks(a0.elapsed_time(a1) / args.e2e_steps, ws)
        ok = bool(np.array_equal(h_perm.numpy(), perm.cpu().numpy()))
        e2e = {"value": job_rate(N, ws, ems / 1e3), "unit": "chars/s",
               "h2d_bytes_per_step": int(chars.numel() + 8 * n + 4 * n),
               "d2h_bytes_per_step": int(8 * n + 16 * args.p),
               "ms_per_step": ems, "result_read_back": ok}
        if ws == 1:
            del d_chars, d_offs, d_lens
            e2e["host_link"] = bench_h2d(args, dev)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline(args.cpu_sample)
        except Exception as ex:  # reported, not fatal
            cpu = {"error": str(ex)[:200]}

    if args.breakdown and rank == 0:
        print_breakdown(stats_all, "pdms")

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "chars/s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "u8", "data": "synthetic",
               "strings_per_s": n * ws / (ms_step / 1e3),
               "config": {"workload": WORKLOAD if (n == N_FULL and args.p == P) else f"pdms_{n}x500_p{args.p}",
                          "strings": n, "chars": N, "partitions": args.p,
                          "D_over_N": D / N, "approx_over_N": Dapprox / N,
                          "l2": "inputs (2.1 GB of chars) larger than L2; no flush",
                          "parallelism": f"replicas x{ws}"},
               "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                            "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                            "frac_of_nominal_8tbs": achieved / 8000.0,
                            "algorithmic_bytes_per_launch": algo, "avg_launch_ms": avg_ms},
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
               "kernels_per_step": sum(v["launches"] for v in stats_all.values()), "round_loop": round_loop,
               "paper_context": {"note": "the paper's own PDMS wall times on SuperMUC-NG (48-core nodes), "
                                         "DNData n/p = 1e5, as chars/s; other hardware, not a target",
                                 "pdms1_4_nodes_192_cores": 1.62e10, "pdms2_4_nodes_192_cores": 1.51e10,
                                 "pdms3_1024_nodes_49152_cores": 2.29e12},
               "kernel_ms_per_step": {k: v["total_ms"] for k, v in stats_all.items()},
               "stages": stage_rooflines({k: v["total_ms"] for k, v in stats_all.items()}, n, D, Dapprox, sum_lcp,
                                         hbm)}
        if ws == 1 and args.workload == "all":
            del chars, offs, lens, perm, lcp, dist_t, approx
            out["batch"] = bench_batch(args, dev, ctx)
            torch.cuda.empty_cache()
            out["char_sampling"] = bench_charsample(args, dev, ctx)
            torch.cuda.empty_cache()
            out["suffix_sort"] = bench_suffix(args, dev, ctx)
            torch.cuda.empty_cache()
            out["config1_plain"] = bench_config1(args, dev, ctx)
            torch.cuda.empty_cache()
            out["config3_suffixes"] = bench_config3(args, dev, ctx)
            torch.cuda.empty_cache()
            out["serving"] = bench_serve(args, dev)
            out["p50_ms"] = out["serving"].get("p50_ms")
            out["p99_ms"] = out["serving"].get("p99_ms")
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def print_breakdown(stats: dict, title: str):
    tot = sum(v["total_ms"] for v in stats.values()) or 1.0
    print(f"-- {title}: {tot:.3f} ms in kernels", file=sys.stderr)
    for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["total_ms"]):
        print(f"{k:18s} launches {v['launches']:6d}  {v['total_ms']:9.3f} ms  {100 * v['total_ms'] / tot:5.1f}%",
              file=sys.stderr)


def bench_batch(args, dev, ctx):
    """4,096 independent instances (sizes log-uniform over 2^6..2^16 strings,
    lengths 8..300 over ACGT, per-instance D/N ratio 0.1..0.9) sorted by one
    sss_sort_batch call per step, against one sss_sort call per instance."""
    import numpy as np
    import torch

    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as sss
    tg = time.perf_counter()
    chars, offs, lens, first = dgc.config4(args.batch_instances)
    torch.cuda.synchronize()
    tg = time.perf_counter() - tg
    m = len(first) - 1
    sizes = np.diff(first).astype(np.int64)
    n = int(first[-1])
    N = int(lens.to(torch.int64).sum().item())
    prm = sss.params()
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    _, _, d = sss.sss_sort_batch(chars, offs, lens, first[:-1], sizes, prm, perm, lcp, want_dist=True, ctx=ctx)
    D = int(d.to(torch.int64).sum().item())
    del d
    arr, _ = sss.instance_table(first[:-1], sizes)
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(p_):
        ctx._check(sss.lib().sss_sort_batch(ctx.h, sss._ptr(chars), chars.numel(), sss._ptr(offs), sss._ptr(lens), n,
                                            arr, m, sss.C.byref(p_), sss._ptr(perm), sss._ptr(lcp), None), ctx.h)

    def timed(p_, steps):
        for _ in range(args.warmup):
            run(p_)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            run(p_)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    # autotune the knobs on a sample of the instances (outside the timed region)
    tuning = None
    if not args.no_tune:
        from paper_2404_16517_gb300 import autotune
        t0 = time.perf_counter()
        best, table = autotune.tune_batch(chars, offs, lens, first[:-1], sizes, max_strings=1 << 22, ctx=ctx)
        ms_default = timed(prm, max(1, args.steps // 2))
        prm_t = sss.params(**best)
        ms_tuned = timed(prm_t, max(1, args.steps // 2))
        if ms_tuned < ms_default:
            prm = prm_t
        tuning = {"chosen": best if ms_tuned < ms_default else "defaults", "candidates": len(table),
                  "sample_strings_max": 1 << 22, "tune_s": time.perf_counter() - t0,
                  "ms_default_knobs": ms_default, "ms_tuned_knobs": ms_tuned,
                  "fastest_on_sample_ms": table[0][0], "slowest_on_sample_ms": table[-1][0]}

    # the whole sort as one CUDA graph launch, against the host-driven round loop
    graph = None
    if not args.no_graph:
        prm_g = sss.params(flags=prm.flags | sss.SSS_FLAG_GRAPH, cta_cap=prm.cta_cap, direct_cap=prm.direct_cap,
                           bucket_target=prm.bucket_target, warp_cap=prm.warp_cap)
        ms_host = timed(prm, max(1, args.steps // 2))
        ms_graph = timed(prm_g, max(1, args.steps // 2))
        graph = {"ms_host_loop": ms_host, "ms_graph": ms_graph, "used": ms_graph < ms_host}
        p_host = perm.clone()
        run(prm_g)
        torch.cuda.synchronize()
        graph["outputs_identical"] = bool(torch.equal(p_host, perm))
        if ms_graph < ms_host:
            prm = prm_g

    def step():
        run(prm)

    # per-kernel launch counts and times from one host-driven pass (kernels
    # inside a graph launch are not timed one by one)
    prm_h = sss.params(flags=prm.flags & ~sss.SSS_FLAG_GRAPH, cta_cap=prm.cta_cap, direct_cap=prm.direct_cap,
                       bucket_target=prm.bucket_target, warp_cap=prm.warp_cap)
    ctx.reset_stats()
    ctx.set_timing(True, "")
    run(prm_h)
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.set_timing(False)
    launches = sum(v["launches"] for v in stats.values())
    if args.breakdown:
        print_breakdown(stats, "batch")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    p_batch = perm.cpu()

    if args.per_instance_steps <= 0:
        per = None
    else:
        per = per_instance_calls(args, ctx, chars, offs, lens, first, perm, lcp, p_batch, prm, e0, e1, st)
    hbm, peak_kind = peaks()
    algo = D + 20 * n
    return {"workload": f"batch_{m}_instances_2^6..2^16_len8..300_ACGT", "instances": m, "strings": n, "chars": N,
            "D_over_N": D / N, "ms_per_step": ms, "chars_per_s": N / (ms / 1e3), "strings_per_s": n / (ms / 1e3),
            # with the graph used a step is one instance-table upload and one graph
            # launch whose nodes run the kernels counted from the host-driven pass
            "gpu_launches_per_step": 1 if (graph and graph["used"]) else launches,
            "kernels_per_step": launches, "tuning": tuning, "graph": graph,
            "per_instance_calls": per,
            "speedup_vs_per_instance": (per["ms_per_step"] / ms) if per else None,
            "outputs_identical": per["outputs_identical"] if per else None,
            "roofline": {"bound": "hbm", "achieved": algo / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": algo / (ms / 1e3) / 1e9 / hbm, "peak_kind": peak_kind,
                         "algorithmic_bytes": algo, "model": "D + 20n (dist chars, views, perm, lcp)"},
            "steps": args.steps, "warmup": args.warmup, "generate_s": tg,
            "l2": "inputs (%.1f GB of chars) larger than L2; no flush" % (N / 1e9)}


def per_instance_calls(args, ctx, chars, offs, lens, first, perm, lcp, p_batch, prm, e0, e1, st):
    """The same instances sorted by one sss_sort call each (p = 1)."""
    import torch

    import paper_2404_16517_gb300 as sss
    m = len(first) - 1
    N = int(lens.to(torch.int64).sum().item())
    perm2 = torch.empty_like(perm)
    lcp2 = torch.empty_like(lcp)
    fi = [int(x) for x in first]

    def per_instance():
        for k in range(m):
            a, b = fi[k], fi[k + 1]
            sss.sss_sort(chars, offs[a:b], lens[a:b], 1, prm, perm2[a:b], lcp2[a:b], ctx=ctx)

    ctx.reset_stats()
    ctx.set_timing(True, "")
    per_instance()
    torch.cuda.synchronize()
    stats1 = ctx.kernel_stats()
    ctx.set_timing(False)
    launches1 = sum(v["launches"] for v in stats1.values())
    per_instance()
    torch.cuda.synchronize()
    steps1 = max(1, min(args.per_instance_steps, 2))
    e0.record(st)
    for _ in range(steps1):
        per_instance()
    e1.record(st)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / steps1
    same = bool(torch.equal(p_batch, perm2.cpu()) and torch.equal(lcp.cpu(), lcp2.cpu()))
    return {"ms_per_step": ms1, "chars_per_s": N / (ms1 / 1e3), "gpu_launches_per_step": launches1,
            "steps": steps1, "outputs_identical": same}


def bench_serve(args, dev):
    """Open-loop Poisson stream of sort requests (sizes lognormal, median 2^14
    strings, sigma 1.5, capped at 2^24; lengths 16..1000 over A-Z; per-request
    copy ratio 0.1..0.9) through the request loop under an HBM budget, at a rate
    of `load` times the saturated rate of a closed-loop warm-up."""
    import numpy as np
    import torch

    import datagen
    import datagen.cuda as dgc
    from paper_2404_16517_gb300.serve import Request, Server, summarize

    def make(count, seed, rid0=0):
        sz, rt, gaps, sd = datagen.config5_requests(count, seed=seed)
        tot = dgc.request_totals(sd, sz)
        return [Request(rid=rid0 + i, n=int(sz[i]), chars=int(tot[i]), seed=int(sd[i]), ratio=float(rt[i]))
                for i in range(count)], gaps

    reqs, gaps = make(args.serve_requests, 5)
    warm, _ = make(args.serve_warmup, 6, rid0=1 << 30)
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = Server(device=dev.index, budget_bytes=budget, slots=args.serve_slots,
                 max_batch_requests=args.serve_max_batch)
    t0 = srv.run_closed_loop(warm)
    sat = summarize(warm, t0)
    lam = args.serve_load * sat["requests_per_s"]
    arrivals = list(np.cumsum(gaps) / lam)
    with srv.sched.cv:  # count the open-loop run only
        srv.sched.n_batches, srv.sched.batch_sizes = 0, []
        srv.sched.gen_ms = srv.sched.sort_ms = 0.0
    t0 = srv.run_open_loop(reqs, arrivals)
    st = summarize(reqs, t0)
    hw = srv.sched.alloc.high_water
    nb = srv.sched.n_batches
    gen_ms, sort_ms = srv.sched.gen_ms, srv.sched.sort_ms
    mean_batch = sum(srv.sched.batch_sizes) / max(1, nb)
    srv.close()
    torch.cuda.synchronize()
    st.update({"workload": f"serve_{args.serve_requests}_requests_lognormal_2^14_s1.5_len16..1000_AZ",
               "lambda_per_s": lam, "load": args.serve_load, "saturated_requests_per_s": sat["requests_per_s"],
               "saturated_chars_per_s": sat["chars_per_s"], "warmup_requests": args.serve_warmup,
               "budget_bytes": budget, "arena_high_water_bytes": hw, "slots": args.serve_slots,
               "batches_total": nb, "mean_batch_requests": mean_batch,
               "device_ms_generate_total": gen_ms, "device_ms_sort_total": sort_ms,
               "max_batch_requests": args.serve_max_batch,
               "latency": "scheduled arrival to batch completion on the device (includes queueing, admission, "
                          "on-device generation of the request's strings, sort)"})
    return st


def bench_charsample(args, dev, ctx):
    """String-based against character-based regular sampling (Section 3.1.2) on a
    set whose distinguishing prefixes are skewed and sort last: 4,194,304
    strings over A-Z; those starting with Z are 1000 characters long and share
    992 of them, the others are 20 uniform characters; p = 16, v = 16.  Reports
    the step time and the characters (approx-truncated) of the largest bucket
    over the mean bucket."""
    import torch

    import datagen.cuda as dgc
    import paper_2404_16517_gb300 as sss
    n, p = args.n, args.p
    chars, offs, lens = dgc.skew_set(6, n)
    N = int(lens.to(torch.int64).sum().item())
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rp, _ = sss.sss_local_sort(chars, offs, lens, p, ctx=ctx)
    out = {"workload": f"skew_{n}x(20|1000, Z-strings share 992)_AZ_p{p}", "strings": n, "chars": N}
    perms = {}
    v = 16
    out["v"] = v
    for name, flags in (("string_based", 0), ("char_based", sss.SSS_FLAG_CHAR_SAMPLING)):
        prm = sss.params(v=v, flags=flags)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        lcp = torch.empty(n, dtype=torch.int32, device=dev)
        ap = torch.empty(n, dtype=torch.int32, device=dev)

        def step():
            sss.sss_sort(chars, offs, lens, p, prm, perm, lcp, out_approx=ap, ctx=ctx)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        # bucket characters from this flag's partition of the approx-truncated runs
        _, bnd = sss.sss_partition(chars, offs, lens, rp, p, trunc=ap, prm=prm, ctx=ctx)
        tl = ap.to(torch.int64)[rp.to(torch.int64)]
        cs = torch.zeros(n + 1, dtype=torch.int64, device=dev)
        cs[1:] = torch.cumsum(tl, 0)
        lo = torch.tensor([i * n // p for i in range(p)], dtype=torch.int64, device=dev)
        b = bnd.to(torch.int64) + lo[:, None]
        per = (cs[b[:, 1:]] - cs[b[:, :-1]]).sum(0)
        Nt = int(tl.sum().item())
        out[name] = {"ms_per_step": ms, "chars_per_s": N / (ms / 1e3),
                     "bucket_chars_max_over_mean": float(per.max().item()) / (Nt / p),
                     "bucket_chars_min_over_mean": float(per.min().item()) / (Nt / p)}
        perms[name] = (perm.clone(), lcp.clone())
    out["outputs_identical"] = bool(torch.equal(perms["string_based"][0], perms["char_based"][0]) and
                                    torch.equal(perms["string_based"][1], perms["char_based"][1]))
    return out


def bench_suffix(args, dev, ctx):
    """Suffix array and LCP array of the 2^22-byte order-2 Markov text of the
    suffix workload (64 symbols, Dirichlet(0.1) rows), all 4,194,304 suffixes
    whole, by sss_suffix_sort (suffix views, no characters copied)."""
    import torch

    import datagen
    import paper_2404_16517_gb300 as sss
    text = torch.from_numpy(datagen.markov_text(3, 1 << 22)).to(dev)
    n = text.numel()
    sa = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)

    def step():
        sss.sss_suffix_sort(text, 0, None, sa, lcp, ctx=ctx)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    l64 = lcp.to(torch.int64)
    out = {"workload": "suffix_array_markov_order2_2^22_sigma64", "text_bytes": n, "ms_per_step": ms,
           "suffixes_per_s": n / (ms / 1e3), "mean_lcp": float(l64.float().mean().item()),
           "max_lcp": int(l64.max().item()), "steps": args.steps}
    # a highly repetitive text: 2^22 copies of one character (prefix doubling over
    # ranks; a direct string sort would read n^2/2 characters)
    rep = torch.full((n,), ord("A"), dtype=torch.uint8, device=dev)
    sss.sss_suffix_sort(rep, 0, None, sa, lcp, ctx=ctx)
    torch.cuda.synchronize()
    e0.record(st)
    sss.sss_suffix_sort(rep, 0, None, sa, lcp, ctx=ctx)
    e1.record(st)
    torch.cuda.synchronize()
    ms_rep = e0.elapsed_time(e1)
    k = torch.arange(n, device=dev, dtype=torch.int64)
    ok = bool(torch.equal(sa.to(torch.int64), n - 1 - k) and torch.equal(lcp.to(torch.int64), k))
    out["one_repeated_character"] = {"text_bytes": n, "ms": ms_rep, "suffixes_per_s": n / (ms_rep / 1e3),
                                     "closed_form_ok": ok}
    return out


def bench_sort_config(args, dev, ctx, workload: str, chars, offs, lens, p: int, note: str, steps: int = 20):
    """Time sss_sort on one more string set (a sub-line of the JSON): L2
    flushed (a 256 MB write) before every step, each step timed by its own CUDA
    events on the context stream, the dominant kernel's roofline and the
    stage-level efficiencies as for the headline.  The local sort's round loop
    runs host-driven and as one graph launch (SSS_FLAG_GRAPH); the faster is
    reported, both are listed."""
    import torch

    import paper_2404_16517_gb300 as sss
    n = lens.numel()
    N = int(lens.to(torch.int64).sum().item())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)
    perm0 = torch.empty(n, dtype=torch.int32, device=dev)
    lcp0 = torch.empty(n, dtype=torch.int32, device=dev)

    def loop_ms(prm_, reps):
        for _ in range(3):
            sss.sss_sort(chars, offs, lens, p, prm_, perm0, lcp0, ctx=ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for i in range(reps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(st)
            sss.sss_sort(chars, offs, lens, p, prm_, perm0, lcp0, ctx=ctx)
            ev[i][1].record(st)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    ms_host = loop_ms(sss.params(), 10)
    ms_graph = loop_ms(sss.params(flags=sss.SSS_FLAG_GRAPH), 10)
    prm = sss.params(flags=sss.SSS_FLAG_GRAPH) if ms_graph < ms_host else sss.params()
    del perm0, lcp0
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    dist_t = torch.empty(n, dtype=torch.int32, device=dev)
    approx = torch.empty(n, dtype=torch.int32, device=dev) if p > 1 else None

    def step(prm_=None):
        sss.sss_sort(chars, offs, lens, p, prm_ or prm, perm, lcp, out_dist=dist_t, out_approx=approx, ctx=ctx)

    for _ in range(args.warmup):
        step()
    # per-kernel times from one host-driven pass (kernels inside a graph launch
    # are not timed one by one)
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_timing(True, "")
    step(sss.params())
    torch.cuda.synchronize()
    stats_all = ctx.kernel_stats()
    ctx.set_timing(False)
    dom = max(stats_all.items(), key=lambda kv: kv[1]["total_ms"])[0]
    D = int(dist_t.to(torch.int64).sum().item())
    Dapprox = int(approx.to(torch.int64).sum().item()) if approx is not None else D
    sum_lcp = int(lcp.to(torch.int64).sum().item())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ctx.reset_stats()
    ctx.set_timing(True, dom)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(st)
        step()
        ev[i][1].record(st)
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.set_timing(False)
    ms_step = statistics.mean(a.elapsed_time(b) for a, b in ev)
    hbm, peak_kind = peaks()
    dstat = stats.get(dom, {"launches": 0, "total_ms": 0.0, "timed": 0})
    per_step = steps
    if dstat["timed"] == 0:  # the dominant kernel ran inside the graph: its host-driven time
        dstat, per_step = stats_all.get(dom), 1
    avg_ms = dstat["total_ms"] / max(1, dstat["timed"])
    algo = algorithmic_bytes(dom, n, N, D, Dapprox, dstat["launches"] / max(1, per_step))
    achieved = algo / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    launches = sum(v["launches"] for v in stats.values()) / steps
    kernels = sum(v["launches"] for v in stats_all.values())
    return {"workload": workload, "strings": n, "chars": N, "partitions": p, "steps": steps,
            "ms_per_step": ms_step, "chars_per_s": N / (ms_step / 1e3), "strings_per_s": n / (ms_step / 1e3),
            "D_over_N": D / max(1, N), "approx_over_N": Dapprox / max(1, N), "gpu_launches_per_step": launches,
            "kernels_per_step": kernels,
            "round_loop": {"ms_host_loop": ms_host, "ms_graph": ms_graph,
                           "used": "graph" if ms_graph < ms_host else "host"},
            "l2": note,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo,
                         "avg_launch_ms": avg_ms},
            "kernel_ms_per_step": {k: v["total_ms"] for k, v in stats_all.items()},
            "stages": stage_rooflines({k: v["total_ms"] for k, v in stats_all.items()}, n, D, Dapprox, sum_lcp,
                                      hbm)}


def bench_config1(args, dev, ctx):
    """65,536 strings x 100 chars (4 templates sharing 42 chars), p = 1: plain
    local sort with LCP array and exact dist."""
    import datagen.cuda as dgc
    chars, offs, lens = dgc.config1()
    return bench_sort_config(args, dev, ctx, "plain_65536x100_AZ_T4_shared42_p1", chars, offs, lens, 1,
                             "inputs (6.6 MB) fit in L2: L2 flushed by a 256 MB write before every step", steps=50)


def bench_config3(args, dev, ctx):
    """2,097,152 suffixes (length <= 256) at distinct random offsets of a
    2^22-byte order-2 Markov text over 64 symbols, p = 64: the full pipeline."""
    import datagen
    import paper_2404_16517_gb300 as sss
    ss = datagen.config3()
    chars, offs, lens = sss.to_device(ss, dev)
    return bench_sort_config(args, dev, ctx, "suffixes_2097152_of_markov2_2^22_sigma64_max256_p64", chars, offs,
                             lens, 64, "the 4 MiB text and the 25 MB of views fit in L2: L2 flushed by a 256 MB "
                                       "write before every step", steps=20)


def bench_h2d(args, dev, nbytes: int = 2 << 30) -> dict:
    """Host link: a 2 GiB copy from pinned host memory to the device split over
    1, 2, 4 and 8 streams, and one copy back (best of three, CUDA events)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h.fill_(65)
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {"bytes": nbytes, "h2d_gbs": {}}
    for ns in (1, 2, 4, 8):
        streams = [torch.cuda.Stream(dev) for _ in range(ns)]
        best = None
        for _ in range(3):
            torch.cuda.synchronize()
            start = torch.cuda.Event(enable_timing=True)
            start.record()
            ends = []
            ch = nbytes // ns
            for i, st in enumerate(streams):
                e1 = torch.cuda.Event(enable_timing=True)
                st.wait_event(start)
                with torch.cuda.stream(st):
                    d[i * ch:(i + 1) * ch].copy_(h[i * ch:(i + 1) * ch], non_blocking=True)
                    e1.record(st)
                ends.append(e1)
            torch.cuda.synchronize()
            # from the common start to the last stream's end
            ms = max(start.elapsed_time(e) for e in ends)
            best = ms if best is None else min(best, ms)
        out["h2d_gbs"][str(ns)] = nbytes / (best / 1e3) / 1e9
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(3):
        torch.cuda.synchronize()
        e0.record()
        h.copy_(d, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    out["d2h_gbs"] = nbytes / (best / 1e3) / 1e9
    return out


def algorithmic_bytes(kernel: str, n: int, N: int, D: int, Dapprox: int, launches_per_step: float) -> float:
    """Minimum bytes a launch of `kernel` must move on this workload."""
    lps = max(launches_per_step, 1.0)
    models = {
        # local sort: every string's distinguishing prefix plus its view and outputs
        "ls_lg_ext": (D + 16 * n) / lps,
        "ls_finish_cta": (D + 24 * n) / lps,
        "pd_hash": (Dapprox / 2 + 32 * n) / lps,
        "d_merge": 32 * n / lps,
        "d_search": 32 * n / lps,
    }
    return float(models.get(kernel, 24 * n / lps))


STAGE_OF = (("ls_", "A"), ("dist", "A"), ("pd_", "B"), ("c_", "C"), ("d2_", "D"), ("d_", "D"))


def stage_rooflines(kernel_ms: dict, n: int, D: int, Dapprox: int, sum_lcp: int, peak_gbs: float) -> dict:
    """Stage-level algorithmic-byte efficiency of one step: each
    stage's kernel time (CUDA events, per step) against the bytes its step must
    move at least.  A: D + 20n (distinguishing prefixes, views, perm and lcp)
    plus 12n for dist; B: sum(approx) + 16n (prefix characters read once, one
    key per string, approx); C: negligible (samples and p^2 searches); D: the
    LCP-compressed records, about sum(approx) - sum(lcp) characters + 8n,
    written by the scatter and read twice by the merge, plus 8n of output."""
    ms = {"A": 0.0, "B": 0.0, "C": 0.0, "D": 0.0, "other": 0.0}
    for k, v in kernel_ms.items():
        st = next((s for pre, s in STAGE_OF if k.startswith(pre)), "other")
        ms[st] += v
    rec = max(0, Dapprox - sum_lcp) + 8 * n
    algo = {"A": D + 32 * n, "B": Dapprox + 16 * n, "C": None, "D": 3 * rec + 8 * n, "other": None}
    out = {}
    for st, t in ms.items():
        a = algo[st]
        gbs = a / (t / 1e3) / 1e9 if (a is not None and t > 0) else None
        out[st] = {"ms": t, "algorithmic_bytes": a, "achieved_gbs": gbs,
                   "frac": gbs / peak_gbs if gbs is not None else None}
    return out


def known_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current library source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("source_hash") == lib_source_hash() and kernel in d.get("kernels", {}):
            return d["kernels"][kernel]
    except Exception:
        pass
    return None


if __name__ == "__main__":
    sys.exit(main())
