"""Autotuner for the collision kernel's launch shape.

The tunable is the thread-block cluster size C (the number of CTAs that share
one cell: the spectral slab per CTA, the exchange volume and the number of
resident clusters all follow from it).  For every velocity-grid class of a
batch (or for one context) it times each compiled C with CUDA events on the
caller's data and keeps the fastest; results are cached in a JSON file keyed
by device name, precision and n.
"""
from __future__ import annotations

import json
import os

from . import fks

# cluster sizes compiled for each (precision, n)
CANDIDATES = {
    (fks.FKS_FP32, 8): [1, 2], (fks.FKS_FP32, 16): [1, 2], (fks.FKS_FP32, 24): [2, 4], (fks.FKS_FP32, 32): [4, 8, 16],
    (fks.FKS_FP64, 8): [1, 2], (fks.FKS_FP64, 16): [2, 4], (fks.FKS_FP64, 24): [4], (fks.FKS_FP64, 32): [8],
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


def tune_batch(batch: "fks.Batch", fs, Qs, precision, reps: int = 3, cache: str | None = DEFAULT_CACHE,
               use_cache: bool = True) -> dict:
    """Choose C for every n class of `batch` (timing batch.collide on fs -> Qs)."""
    import torch
    data = _load(cache) if cache else {}
    chosen = {}
    for n in sorted(set(batch.n)):
        key = _key(torch, precision, n)
        if use_cache and key in data:
            batch.set_cluster_size(n, int(data[key]["C"]))
            chosen[n] = int(data[key]["C"])
            continue
        timings = {}
        for C in CANDIDATES[(precision, n)]:
            batch.set_cluster_size(n, C)
            timings[C] = _time(torch, lambda: batch.collide(fs, Qs), reps)
        best = min(timings, key=timings.get)
        batch.set_cluster_size(n, best)
        chosen[n] = best
        data[key] = {"C": best, "ms": {str(c): t for c, t in timings.items()}}
    if cache:
        _save(cache, data)
    return chosen


def tune_context(ctx: "fks.Context", f, Q, reps: int = 3, cache: str | None = DEFAULT_CACHE,
                 use_cache: bool = True) -> int:
    """Choose C for one context (timing ctx.collide on f -> Q)."""
    import torch
    precision = ctx.cfg.precision
    n = ctx.cfg.n
    data = _load(cache) if cache else {}
    key = _key(torch, precision, n) + f"|cells{ctx.ncells}"
    if use_cache and key in data:
        ctx.set_cluster_size(int(data[key]["C"]))
        return int(data[key]["C"])
    timings = {}
    for C in CANDIDATES[(precision, n)]:
        ctx.set_cluster_size(C)
        timings[C] = _time(torch, lambda: ctx.collide(f, Q), reps)
    best = min(timings, key=timings.get)
    ctx.set_cluster_size(best)
    data[key] = {"C": best, "ms": {str(c): t for c, t in timings.items()}}
    if cache:
        _save(cache, data)
    return best
