"""Autotuner for the sorter's tuning knobs (sss_params: cta_cap, direct_cap,
bucket_target, warp_cap, merge_ms).

The knobs set the local sort's size classes: segments of at most warp_cap
strings are finished by one warp, up to cta_cap by one CTA, up to direct_cap by
one whole-segment CTA sort after the reference split, and larger segments are
split by sampled partition into range buckets of about bucket_target strings.
They change speed, never results.  The tuner times candidate settings on a
sample of the caller's own workload (CUDA events on the context stream, median
of a few runs after a warm-up) and returns the fastest; results can be cached in
a JSON file keyed by the GPU name and a coarse signature of the workload.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

import torch

from . import Context, context, instance_table, lib, params, sss_sort, _ptr

DEFAULT_GRID = {
    "cta_cap": [512, 1024, 2048],
    "direct_cap": [2048, 4096, 8192],
    "bucket_target": [1024, 2048, 4096],
    "warp_cap": [16, 32],
}


def candidates(grid: dict | None = None) -> list[dict]:
    """Every valid combination of the grid (direct_cap >= cta_cap)."""
    grid = grid or DEFAULT_GRID
    keys = sorted(grid)
    out = []
    for vals in itertools.product(*(grid[k] for k in keys)):
        c = dict(zip(keys, vals))
        if c.get("direct_cap", 8192) < c.get("cta_cap", 2048):
            continue
        out.append(c)
    return out


def _time(fn, ctx: Context, reps: int) -> float:
    st = torch.cuda.current_stream()
    fn()
    ctx.sync()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def sample_instances(first, sizes, max_strings: int, seed: int = 0):
    """Instances in a seeded random order until about max_strings strings are
    taken, so the sample keeps the size mix.  Returns (first, sizes) of the
    sample in table order."""
    import numpy as np
    m = len(sizes)
    order = np.random.default_rng(seed).permutation(m)
    take, tot = [], 0
    for i in order:
        if take and tot + int(sizes[i]) > max_strings:
            continue
        take.append(int(i))
        tot += int(sizes[i])
        if tot >= max_strings:
            break
    take.sort()
    return [int(first[i]) for i in take], [int(sizes[i]) for i in take]


def tune_batch(chars, offs, lens, first, sizes, grid: dict | None = None, max_strings: int = 1 << 22,
               reps: int = 3, ctx: Context | None = None, base=None):
    """Time sss_sort_batch over a sample of the instances for every candidate;
    returns (best knob dict, [(ms, knobs), ...] sorted fastest first)."""
    ctx = ctx or context(chars.device.index)
    f_s, n_s = sample_instances(first, sizes, max_strings)
    n = lens.numel()
    perm = torch.empty(n, dtype=torch.int32, device=chars.device)
    lcp = torch.empty(n, dtype=torch.int32, device=chars.device)
    arr, m = instance_table(f_s, n_s)
    results = []
    for c in candidates(grid):
        prm = _with(base, c)

        def run():
            ctx._check(lib().sss_sort_batch(ctx.h, _ptr(chars), chars.numel(), _ptr(offs), _ptr(lens), n, arr, m,
                                            _byref(prm), _ptr(perm), _ptr(lcp), None), ctx.h)
        results.append((_time(run, ctx, reps), c))
    results.sort(key=lambda x: x[0])
    return results[0][1], results


def tune_sort(chars, offs, lens, p: int, grid: dict | None = None, reps: int = 3, ctx: Context | None = None,
              base=None):
    """Time sss_sort (p partitions) for every candidate; same return value."""
    ctx = ctx or context(chars.device.index)
    n = lens.numel()
    perm = torch.empty(n, dtype=torch.int32, device=chars.device)
    lcp = torch.empty(n, dtype=torch.int32, device=chars.device)
    results = []
    for c in candidates(grid):
        prm = _with(base, c)
        results.append((_time(lambda: sss_sort(chars, offs, lens, p, prm, perm, lcp, ctx=ctx), ctx, reps), c))
    results.sort(key=lambda x: x[0])
    return results[0][1], results


def _with(base, knobs: dict):
    prm = params()
    if base is not None:
        for name, _ in base._fields_:
            setattr(prm, name, getattr(base, name))
    for k, v in knobs.items():
        setattr(prm, k, int(v))
    return prm


def _byref(prm):
    import ctypes
    return ctypes.byref(prm)


def signature(kind: str, n: int, total_chars: int, m: int = 1) -> str:
    """Coarse workload key: kind, and the powers of two of strings, characters
    and instances."""
    def lg(x):
        return max(0, int(x).bit_length() - 1)
    return f"{kind}:n2^{lg(n)}:N2^{lg(total_chars)}:m2^{lg(m)}"


def cached(path: str, key: str, device_name: str | None = None):
    """Knobs stored for (this GPU, key) in the JSON cache at path, or None."""
    device_name = device_name or torch.cuda.get_device_name()
    try:
        with open(path) as f:
            d = json.load(f)
        return d.get(device_name, {}).get(key)
    except (OSError, ValueError):
        return None


def store(path: str, key: str, knobs: dict, device_name: str | None = None):
    device_name = device_name or torch.cuda.get_device_name()
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        d = {}
    d.setdefault(device_name, {})[key] = knobs
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
