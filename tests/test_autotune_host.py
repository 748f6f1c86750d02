"""Host logic of the cluster-size autotuner (paper_1701_01608_gb300/autotune.py): its candidate
table against the instantiations compiled in the library, the choice of the fastest candidate and
the JSON cache, with the device timing replaced by a table of times."""
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
        out.setdefault(int(n), []).append(int(c))
    return {n: sorted(cs) for n, cs in out.items()}


@pytest.mark.parametrize("precision,fname", [(fks.FKS_FP32, "fks_collide_f32.cu"), (fks.FKS_FP64, "fks_collide_f64.cu")])
def test_candidates_are_the_compiled_variants(precision, fname):
    compiled = _compiled(fname)
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

    def set_cluster_size(self, C):
        self.C = C
        self.history.append(C)

    def collide(self, f, Q):
        pass


class _Batch:
    def __init__(self, ns):
        self.n = list(ns)
        self.C = {}

    def set_cluster_size(self, n, C):
        self.C[n] = C

    def collide(self, fs, Qs):
        pass


@pytest.fixture
def fake_timing(monkeypatch):
    """_time returns times[(n, C)] for the cluster size currently set on the tuned object."""
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
    fake_timing["times"] = {(32, 4): 3.0, (32, 8): 1.5, (32, 16): 2.0}
    assert A.tune_context(ctx, None, None, cache=cache) == 8
    assert ctx.C == 8 and sorted(set(ctx.history)) == [4, 8, 16]
    calls = fake_timing["calls"]
    # second call: read from the cache, nothing timed
    ctx2 = _Ctx(fks.FKS_FP32, 32)
    fake_timing["obj"] = ctx2
    assert A.tune_context(ctx2, None, None, cache=cache) == 8
    assert fake_timing["calls"] == calls and ctx2.history == [8]
    # use_cache=False re-times and follows new timings
    fake_timing["times"][(32, 16)] = 0.5
    assert A.tune_context(ctx2, None, None, cache=cache, use_cache=False) == 16


def test_tune_batch_per_class(tmp_path, fake_timing):
    cache = str(tmp_path / "tune.json")
    b = _Batch([16, 32, 16, 24])
    last = {}

    orig = b.set_cluster_size

    def record(n, C):
        last["nc"] = (n, C)
        orig(n, C)

    b.set_cluster_size = record
    fake_timing["obj"] = b
    fake_timing["current"] = lambda: last["nc"]
    fake_timing["times"] = {(16, 1): 2.0, (16, 2): 1.0, (24, 2): 1.0, (24, 4): 3.0,
                            (32, 4): 5.0, (32, 8): 4.0, (32, 16): 6.0}
    chosen = A.tune_batch(b, None, None, fks.FKS_FP32, cache=cache)
    assert chosen == {16: 2, 24: 2, 32: 8}
    assert b.C == chosen
    assert os.path.exists(cache)


def test_corrupt_cache_is_ignored(tmp_path, fake_timing):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    ctx = _Ctx(fks.FKS_FP64, 16)
    fake_timing["obj"] = ctx
    fake_timing["times"] = {(16, 2): 1.0, (16, 4): 2.0}
    assert A.tune_context(ctx, None, None, cache=str(cache)) == 2
