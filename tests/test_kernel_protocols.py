"""Race and deadlock check of the synchronisation protocols of the cluster kernels, on the CPU.

compute-sanitizer's race and sync checks are not available here, so each kernel's protocol is written
out as the sequence of barriers, mbarrier waits, bulk copies and shared-memory accesses that its code
executes (csrc/fks_collide.cuh: collide_kernel, its staged and its split-pencil exchange;
csrc/fks_bgk.cu: bgk_cluster_kernel) and run under many
seeded schedules by a vector-clock model (tests/harness/protocol_model.py).  The written-out
protocols follow the kernels statement by statement; each test also plants a plausible mistake
(a barrier dropped or moved) and checks that the model reports it, so that a model too weak to see a
race cannot pass silently."""
import os
import sys

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "harness"))
from protocol_model import run  # noqa: E402

TPC = 2   # modelled threads per CTA: thread 0 = tid 0 (issues the table copies, warp 0), thread 1 = the rest


def collide_program(c, i, C, cells, M, mutate=None):
    """collide_kernel<T, N, C>: forward transform through W staging and remote f^ stores, then per
    direction the x-pass (own block into W, peers' blocks into staging S), bulk copies S -> peer W
    completing on the peer's exchange mbarrier, y-pass in place, z-pass; the loss pass ends with the
    cluster reduction of the moment partials.  Locations: ('W', cta, source slot), ('S', cta, peer),
    ('Fh', cta), ('Tb', cta), ('red', cta)."""
    P = []
    acc = lambda loc, k, e, s: P.append(("acc", loc, k, e, s))
    t0 = i == 0
    if t0 and cells:
        P.append(("tma", (cells[0], 0)))      # slab 0 of the first cell, before the init barrier
    P += [("carrive",), ("cwait",)]           # every CTA is running before any remote access
    for ci, cell in enumerate(cells):
        nxt = cells[ci + 1] if ci + 1 < len(cells) else None
        P.append(("sync",))                   # gather offsets along z written
        for s in range(C):                    # F1: z-R2C into the staging (first part of W)
            acc(("W", c, s), "w", ("F", cell), "F1")
        if mutate != "no_sync_after_staging":
            P.append(("sync",))
        for s in range(C):                    # F2: y-FFT from the staging, scatter to the ky owners
            acc(("W", c, s), "r", ("F", cell), "F2")
        for d in range(C):
            acc(("Fh", d), "w", ("F", cell), "F2")
        P += [("carrive",), ("cwait",)]
        acc(("Fh", c), "r", ("F", cell), "F4")     # F4: x-FFT in place
        acc(("Fh", c), "w", ("F", cell), "F4")
        P.append(("sync",))
        P.append(("carrive",))                # matches the wait before the first exchange
        for p in range(M + 1):
            loss = p == M
            P.append(("twait",))
            acc(("Tb", c), "r", ("slab", (cell, p)), "x")
            acc(("Fh", c), "r", ("F", cell), "x")
            if mutate != "no_wait_before_stores":
                P.append(("cwait",))
            acc(("W", c, c), "w", ("dir", cell, p), "x")
            for d in range(C):
                if d != c:
                    acc(("S", c, d), "w", ("dir", cell, p), "x")
            if mutate == "no_wait_before_stores":
                P.append(("cwait",))
            P.append(("sync",))
            if i == 1:                        # the issuing threads (tid = peer rank)
                for d in range(C):
                    if d != c:
                        P.append(("bulk", d, ("S", c, d), ("W", d, c), ("dir", cell, p)))
            if t0:
                if not loss:
                    P.append(("tma", (cell, p + 1)))
                elif nxt is not None:
                    P.append(("tma", (nxt, 0)))
            if C > 1:
                P.append(("xwait", C - 1))
            for s in range(C):                # y-pass in place over every source slot
                acc(("W", c, s), "r", ("dir", cell, p), "y")
                acc(("W", c, s), "w", ("dir", cell, p), "y")
            if mutate != "no_sync_before_z":
                P.append(("sync",))
            for s in range(C):
                acc(("W", c, s), "r", ("dir", cell, p), "z")
            if not loss:
                P.append(("carrive",))
            else:
                P.append(("sync",))           # warp partials staged
                if t0:
                    acc(("red", c), "w", ("cell", cell), "ep")
                P += [("carrive",), ("cwait",)]
                if t0:
                    for d in range(C):
                        acc(("red", d), "r", ("cell", cell), "ep2")
                if mutate != "no_final_barrier":
                    P += [("carrive",), ("cwait",)]
                else:
                    P += [("sync",)]
    return P


def collide_direct_program(c, i, C, cells, M, tables=True, mutate=None):
    """collide_kernel, split-pencil path (double-float): forward transform as above, then per direction p
    the x-pass stores straight into block c of every CTA's W[p mod 2] (DSMEM), one cluster barrier, the
    next table slab (staged tables only), y-pass in place, z-pass; no staging blocks, no bulk copies.
    Locations: ('W', cta, buffer, source slot), ('Fh', cta), ('Tb', cta), ('red', cta)."""
    P = []
    acc = lambda loc, k, e, s: P.append(("acc", loc, k, e, s))
    t0 = i == 0
    nbuf = 1 if mutate == "single_w_buffer" else 2
    if t0 and cells and tables:
        P.append(("tma", (cells[0], 0)))
    P += [("carrive",), ("cwait",)]
    for ci, cell in enumerate(cells):
        nxt = cells[ci + 1] if ci + 1 < len(cells) else None
        P.append(("sync",))
        for s in range(C):                    # F1: staging in the first W buffer
            acc(("W", c, 0, s), "w", ("F", cell), "F1")
        P.append(("sync",))
        for s in range(C):
            acc(("W", c, 0, s), "r", ("F", cell), "F2")
        for d in range(C):
            acc(("Fh", d), "w", ("F", cell), "F2")
        P += [("carrive",), ("cwait",)]
        acc(("Fh", c), "r", ("F", cell), "F4")
        acc(("Fh", c), "w", ("F", cell), "F4")
        P.append(("sync",))
        for p in range(M + 1):
            loss = p == M
            b = p % nbuf
            if tables:
                P.append(("twait",))
                acc(("Tb", c), "r", ("slab", (cell, p)), "x")
            acc(("Fh", c), "r", ("F", cell), "x")
            for d in range(C):                # block c of every CTA's W[b]
                acc(("W", d, b, c), "w", ("dir", cell, p), "x")
            if mutate != "no_barrier_after_stores":
                P += [("carrive",), ("cwait",)]
            if tables and t0:
                if not loss:
                    P.append(("tma", (cell, p + 1)))
                elif nxt is not None:
                    P.append(("tma", (nxt, 0)))
            for s in range(C):
                acc(("W", c, b, s), "r", ("dir", cell, p), "y")
                acc(("W", c, b, s), "w", ("dir", cell, p), "y")
            P.append(("sync",))
            for s in range(C):
                acc(("W", c, b, s), "r", ("dir", cell, p), "z")
            if mutate == "no_barrier_after_stores":
                P += [("carrive",), ("cwait",)]   # the same barrier count, too late
            if loss:
                P.append(("sync",))
                if t0:
                    acc(("red", c), "w", ("cell", cell), "ep")
                P += [("carrive",), ("cwait",)]
                if t0:
                    for d in range(C):
                        acc(("red", d), "r", ("cell", cell), "ep2")
                P += [("carrive",), ("cwait",)]
    return P


def bgk_program(c, i, CL, cells, mutate=None):
    """bgk_cluster_kernel<float, 32, 4>: per cell the gather tables, the loads, the moment partials
    (warp partials in redw, the CTA's in red[parity]), the cluster barrier, warp 0's serial phase
    (every CTA's red[parity] over distributed shared memory; Maxwellian factors and mu), the output."""
    P = []
    acc = lambda loc, k, e, s: P.append(("acc", loc, k, e, s))
    w0 = i == 0
    for k, cell in enumerate(cells):
        par = k & 1 if mutate != "single_partials_buffer" else 0
        P.append(("sync",))
        acc(("src", c), "w", ("cell", cell), "st")
        P.append(("sync",))
        acc(("src", c), "r", ("cell", cell), "ld")
        acc(("redw", c), "w", ("cell", cell), "m")
        P.append(("sync",))
        if w0:
            acc(("redw", c), "r", ("cell", cell), "m2")
            acc(("red", c, par), "w", ("cell", cell), "m2")
        P += [("carrive",), ("cwait",)]
        if w0:
            for d in range(CL):
                acc(("red", d, par), "r", ("cell", cell), "ser")
            acc(("G", c), "w", ("cell", cell), "ser")
        if mutate != "no_sync_before_output":
            P.append(("sync",))
        acc(("G", c), "r", ("cell", cell), "out")
    P += [("carrive",), ("cwait",)]
    return P


def _failures(make, nctas, seeds):
    progs = [make(t // TPC, t % TPC) for t in range(nctas * TPC)]
    bad = []
    for s in range(seeds):
        r = run(progs, nctas, TPC, s)
        if r["deadlock"] or r["races"]:
            bad.append((s, r["deadlock"], r["races"][:2]))
    return bad


@pytest.mark.parametrize("C,M,ncells", [(1, 2, 2), (2, 1, 3), (4, 3, 2), (8, 2, 2)])
def test_collide_kernel_protocol_is_race_and_deadlock_free(C, M, ncells):
    cells = list(range(ncells))
    bad = _failures(lambda c, i: collide_program(c, i, C, cells, M), C, seeds=60)
    assert not bad, bad[0]


@pytest.mark.parametrize("mutate", ["no_sync_after_staging", "no_wait_before_stores", "no_sync_before_z",
                                    "no_final_barrier"])
def test_collide_protocol_model_sees_planted_mistakes(mutate):
    cells = [0, 1]
    bad = _failures(lambda c, i: collide_program(c, i, 4, cells, 2, mutate), 4, seeds=30)
    assert len(bad) >= 25, mutate


@pytest.mark.parametrize("tables", [True, False])
@pytest.mark.parametrize("C,M,ncells", [(1, 2, 2), (2, 1, 3), (4, 3, 2), (8, 2, 2)])
def test_collide_direct_protocol_is_race_and_deadlock_free(C, M, ncells, tables):
    cells = list(range(ncells))
    bad = _failures(lambda c, i: collide_direct_program(c, i, C, cells, M, tables), C, seeds=60)
    assert not bad, bad[0]


@pytest.mark.parametrize("mutate", ["single_w_buffer", "no_barrier_after_stores"])
def test_collide_direct_protocol_model_sees_planted_mistakes(mutate):
    bad = _failures(lambda c, i: collide_direct_program(c, i, 4, [0, 1], 3, True, mutate), 4, seeds=30)
    assert len(bad) >= 25, (mutate, len(bad))


@pytest.mark.parametrize("ncells", [1, 2, 5])
def test_bgk_cluster_kernel_protocol_is_race_and_deadlock_free(ncells):
    cells = list(range(ncells))
    bad = _failures(lambda c, i: bgk_program(c, i, 4, cells), 4, seeds=100)
    assert not bad, bad[0]


@pytest.mark.parametrize("mutate", ["single_partials_buffer", "no_sync_before_output"])
def test_bgk_protocol_model_sees_planted_mistakes(mutate):
    bad = _failures(lambda c, i: bgk_program(c, i, 4, [0, 1, 2], mutate), 4, seeds=60)
    assert len(bad) >= 1, mutate


def test_a_barrier_count_mismatch_is_a_deadlock():
    """One CTA skipping a cluster barrier phase: the model reports the hang."""
    def make(c, i):
        P = collide_program(c, i, 2, [0], 1)
        if c == 1:
            P = [op for op in P if op[0] != "cwait"][:]   # never waits: its peers' waits still complete,
            P = P[:-1]                                       # but it also drops its last arrive
        return P
    progs = [make(t // TPC, t % TPC) for t in range(2 * TPC)]
    with pytest.raises(AssertionError):
        run(progs, 2, TPC, 0)   # arrive twice without a wait: caught as a protocol error
