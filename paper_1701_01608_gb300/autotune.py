"""Autotuner for the collision kernel's launch shape and radix schedule.

Two tunables per (precision, n):
  - the thread-block cluster size C (the number of CTAs that share one cell: the
    spectral slab per CTA, the exchange volume and the number of resident
    clusters follow from it);
  - the radix schedule of the length-n transforms: the top radix of the
    register FFT (0 = the default schedule 32 = 4 x 8, 24 = 3 x 8, 16 = 4 x 4;
    alternatives 2, 4 or 8), which changes the butterfly structure, the twiddle
    count and the register footprint of every pass.
For every velocity-grid class of a batch (or for one context) it times each
compiled (C, radix) with CUDA events on the caller's data and keeps the fastest;
results are cached in a JSON file keyed by device name, precision and n.
"""
from __future__ import annotations

import json
import os

from . import fks

# (cluster size, top radix) pairs compiled for each (precision, n); radix 0 = the default schedule
CANDIDATES = {
    (fks.FKS_FP32, 8): [(1, 0), (2, 0)],
    (fks.FKS_FP32, 16): [(1, 0), (2, 0), (1, 2), (1, 8)],
    (fks.FKS_FP32, 24): [(2, 0), (4, 0), (2, 2), (2, 4), (2, 8)],
    (fks.FKS_FP32, 32): [(4, 0), (8, 0), (16, 0), (8, 2), (8, 8)],
    (fks.FKS_FP64, 8): [(1, 0), (2, 0)],
    (fks.FKS_FP64, 16): [(2, 0), (4, 0)],
    (fks.FKS_FP64, 24): [(4, 0)],
    (fks.FKS_FP64, 32): [(8, 0)],
}

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "autotune.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _key(torch, precision, n):
    return f"{torch.cuda.get_device_name()}|{'fp64' if precision == fks.FKS_FP64 else 'fp32'}|n{n}"


def _time(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def _label(C, radix):
    return f"C{C}/r{radix}"


def _cached(entry):
    """(C, radix) of a cache entry (entries written before the radix dimension hold C alone)."""
    return int(entry["C"]), int(entry.get("radix", 0))


def tune_batch(batch: "fks.Batch", fs, Qs, precision, reps: int = 3, cache: str | None = DEFAULT_CACHE,
               use_cache: bool = True) -> dict:
    """Choose (C, radix) for every n class of `batch` (timing batch.collide on fs -> Qs); returns
    {n: (C, radix)}."""
    import torch
    data = _load(cache) if cache else {}
    chosen = {}
    for n in sorted(set(batch.n)):
        key = _key(torch, precision, n)
        if use_cache and key in data:
            C, r = _cached(data[key])
            batch.set_schedule(n, C, r)
            chosen[n] = (C, r)
            continue
        timings = {}
        for C, r in CANDIDATES[(precision, n)]:
            batch.set_schedule(n, C, r)
            timings[(C, r)] = _time(torch, lambda: batch.collide(fs, Qs), reps)
        best = min(timings, key=timings.get)
        batch.set_schedule(n, *best)
        chosen[n] = best
        data[key] = {"C": best[0], "radix": best[1], "ms": {_label(*k): t for k, t in timings.items()}}
    if cache:
        _save(cache, data)
    return chosen


def tune_context(ctx: "fks.Context", f, Q, reps: int = 3, cache: str | None = DEFAULT_CACHE,
                 use_cache: bool = True) -> tuple:
    """Choose (C, radix) for one context (timing ctx.collide on f -> Q)."""
    import torch
    precision = ctx.cfg.precision
    n = ctx.cfg.n
    data = _load(cache) if cache else {}
    key = _key(torch, precision, n) + f"|cells{ctx.ncells}"
    if use_cache and key in data:
        C, r = _cached(data[key])
        ctx.set_schedule(C, r)
        return (C, r)
    timings = {}
    for C, r in CANDIDATES[(precision, n)]:
        ctx.set_schedule(C, r)
        timings[(C, r)] = _time(torch, lambda: ctx.collide(f, Q), reps)
    best = min(timings, key=timings.get)
    ctx.set_schedule(*best)
    data[key] = {"C": best[0], "radix": best[1], "ms": {_label(*k): t for k, t in timings.items()}}
    if cache:
        _save(cache, data)
    return best
