"""Host logic of the cluster-size autotuner (paper_1701_01608_gb300/autotune.py): its candidate
table against the instantiations compiled in the library, the choice of the fastest candidate and
the JSON cache, with the device timing replaced by a table of times."""
import json
import os
import re

import pytest

from paper_1701_01608_gb300 import autotune as A
from paper_1701_01608_gb300 import fks

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1701_01608_gb300", "csrc")


def _compiled(fname):
    """(n, C) pairs of the `case n * 16 + C: return variant<n, C>` lines of a variant table."""
    text = open(os.path.join(CSRC, fname)).read()
    pairs = re.findall(r"case\s+(\d+)\s*\*\s*16\s*\+\s*(\d+)\s*:\s*return\s+variant<(\d+),\s*(\d+)>", text)
    out = {}
    for n, c, n2, c2 in pairs:
        assert (n, c) == (n2, c2), "case label and instantiation disagree"
        out.setdefault(int(n), []).append((int(c), 0))
    return out


def _compiled_radix(fname):
    """(n, C, radix) of the `case (n * 16 + C) * 16 + R: return collide_variant<float, n, C, float, R>` lines."""
    text = open(os.path.join(CSRC, fname)).read()
    rows = re.findall(r"case\s+\((\d+)\s*\*\s*16\s*\+\s*(\d+)\)\s*\*\s*16\s*\+\s*(\d+)\s*:\s*"
                      r"return\s+collide_variant<float,\s*(\d+),\s*(\d+),\s*float,\s*(\d+)>", text)
    out = {}
    for n, c, r, n2, c2, r2 in rows:
        assert (n, c, r) == (n2, c2, r2), "case label and instantiation disagree"
        out.setdefault(int(n), []).append((int(c), int(r)))
    return out


@pytest.mark.parametrize("precision", [fks.FKS_FP32, fks.FKS_FP64])
def test_candidates_are_the_compiled_variants(precision):
    if precision == fks.FKS_FP32:
        compiled = _compiled("fks_collide_f32.cu")
        radix = _compiled_radix("fks_collide_f32_radix.cu")
        assert radix, "no radix variants found"
        for n, rows in radix.items():
            compiled.setdefault(n, []).extend(rows)
    else:
        compiled = _compiled("fks_collide_f64.cu")
    compiled = {n: sorted(v) for n, v in compiled.items()}
    tuned = {n: sorted(cs) for (p, n), cs in A.CANDIDATES.items() if p == precision}
    assert tuned == compiled


class _Cfg:
    def __init__(self, precision, n):
        self.precision, self.n = precision, n


class _Ctx:
    """Stands in for fks.Context: records the cluster size set by the tuner."""
    def __init__(self, precision, n, ncells=64):
        self.cfg = _Cfg(precision, n)
        self.ncells = ncells
        self.C = None
        self.history = []

    def set_schedule(self, C, radix=0):
        self.C = (C, radix)
        self.history.append(self.C)

    def collide(self, f, Q):
        pass


class _Batch:
    def __init__(self, ns):
        self.n = list(ns)
        self.C = {}

    def set_schedule(self, n, C, radix=0):
        self.C[n] = (C, radix)

    def collide(self, fs, Qs):
        pass


@pytest.fixture
def fake_timing(monkeypatch):
    """_time returns times[(n, (C, radix))] for the schedule currently set on the tuned object."""
    state = {"obj": None, "times": {}, "calls": 0}

    def fake_time(torch, fn, reps):
        state["calls"] += 1
        o = state["obj"]
        if isinstance(o, _Ctx):
            return state["times"][(o.cfg.n, o.C)]
        # batch: the class being timed is the one whose size changed last
        return state["times"][state["current"]()]

    monkeypatch.setattr(A, "_time", fake_time)
    monkeypatch.setattr(A, "_key", lambda torch, precision, n: f"dev|{precision}|n{n}")
    return state


def test_tune_context_picks_fastest_and_caches(tmp_path, fake_timing):
    cache = str(tmp_path / "tune.json")
    ctx = _Ctx(fks.FKS_FP32, 32)
    fake_timing["obj"] = ctx
    fake_timing["times"] = {(32, (4, 0)): 3.0, (32, (8, 0)): 1.5, (32, (16, 0)): 2.0, (32, (8, 2)): 1.8,
                            (32, (8, 8)): 1.2}
    assert A.tune_context(ctx, None, None, cache=cache) == (8, 8)
    assert ctx.C == (8, 8) and sorted(set(ctx.history)) == sorted(A.CANDIDATES[(fks.FKS_FP32, 32)])
    calls = fake_timing["calls"]
    # second call: read from the cache (the radix recorded), nothing timed
    ctx2 = _Ctx(fks.FKS_FP32, 32)
    fake_timing["obj"] = ctx2
    assert A.tune_context(ctx2, None, None, cache=cache) == (8, 8)
    assert fake_timing["calls"] == calls and ctx2.history == [(8, 8)]
    entry = next(iter(json.load(open(cache)).values()))
    assert entry["radix"] == 8 and set(entry["ms"]) == {"C4/r0", "C8/r0", "C16/r0", "C8/r2", "C8/r8"}
    # use_cache=False re-times and follows new timings
    fake_timing["times"][(32, (16, 0))] = 0.5
    assert A.tune_context(ctx2, None, None, cache=cache, use_cache=False) == (16, 0)


def test_cache_entries_without_radix_read_as_default(tmp_path, fake_timing):
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({"dev|1|n32|cells64": {"C": 4, "ms": {}}}))
    ctx = _Ctx(fks.FKS_FP32, 32)
    fake_timing["obj"] = ctx
    assert A.tune_context(ctx, None, None, cache=str(cache)) == (4, 0)


def test_tune_batch_per_class(tmp_path, fake_timing):
    cache = str(tmp_path / "tune.json")
    b = _Batch([16, 32, 16, 24])
    last = {}

    orig = b.set_schedule

    def record(n, C, radix=0):
        last["nc"] = (n, (C, radix))
        orig(n, C, radix)

    b.set_schedule = record
    fake_timing["obj"] = b
    fake_timing["current"] = lambda: last["nc"]
    t = {}
    for n in (16, 24, 32):
        for k, cand in enumerate(A.CANDIDATES[(fks.FKS_FP32, n)]):
            t[(n, cand)] = 5.0 + k
    t[(16, (2, 0))] = 1.0
    t[(24, (2, 8))] = 1.0
    t[(32, (8, 0))] = 1.0
    fake_timing["times"] = t
    chosen = A.tune_batch(b, None, None, fks.FKS_FP32, cache=cache)
    assert chosen == {16: (2, 0), 24: (2, 8), 32: (8, 0)}
    assert b.C == chosen
    assert os.path.exists(cache)


def test_corrupt_cache_is_ignored(tmp_path, fake_timing):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    ctx = _Ctx(fks.FKS_FP64, 16)
    fake_timing["obj"] = ctx
    fake_timing["times"] = {(16, (2, 0)): 1.0, (16, (4, 0)): 2.0}
    assert A.tune_context(ctx, None, None, cache=str(cache)) == (2, 0)
