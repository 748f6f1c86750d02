"""Vector-clock model of the synchronisation protocol of a thread-block-cluster kernel.

A kernel's protocol is written as one list of operations per modelled thread (a CTA is modelled by
a few threads that stand for its warps; thread 0 of a CTA is the one that issues its table copies).
A seeded random scheduler runs the lists with the blocking semantics of the hardware primitives the
kernels use, and every shared-memory access is checked against the earlier ones with vector clocks.

Operations:
  ('carrive',) / ('cwait',)       cluster barrier (barrier.cluster.arrive / wait): all threads of all
                                  CTAs, phases in order; a wait returns once every thread has arrived
                                  for that phase, and joins their clocks
  ('sync',)                       CTA barrier (__syncthreads)
  ('tma', tag)                    bulk copy of a table slab into this CTA's slab buffer ('Tb', cta),
                                  completing on the CTA's table mbarrier
  ('twait',)                      wait for the next table copy of this CTA (mbarrier phase order)
  ('bulk', dst, src_loc, dst_loc, epoch)
                                  bulk copy shared::cta -> shared::cluster into CTA dst, completing
                                  on dst's exchange mbarrier; the copy engine reads src_loc and writes
                                  dst_loc when it completes
  ('xwait', ncopies)              wait for the next exchange phase of this CTA: ncopies copies
  ('acc', loc, kind, epoch, stage)
                                  shared-memory access, kind 'r' or 'w'

A race is a pair of accesses to one location, at least one a write, that happens-before does not
order, unless both belong to the same (epoch, stage): those touch disjoint elements by construction
(different threads' pencils of one pass).  Locations are tuples whose second entry is the CTA that owns
the memory; an access by another CTA (or by a copy engine) must also happen before that CTA exits,
else it would reach the shared memory of a finished CTA.  A deadlock is a state where no thread can
run but some have not finished (a barrier-count or copy-count mismatch: a hang on the GPU).
"""
from __future__ import annotations

import random


class _VC:
    __slots__ = ("v",)

    def __init__(self, n):
        self.v = [0] * n

    def copy(self):
        c = _VC(0)
        c.v = self.v[:]
        return c

    def join(self, o):
        self.v = [a if a >= b else b for a, b in zip(self.v, o.v)]


def run(programs, nctas: int, tpc: int, seed: int) -> dict:
    """Run `programs` (nctas * tpc lists, thread t in CTA t // tpc) under one seeded schedule.
    Returns {"deadlock": None or {thread: pending op}, "races": [...]}."""
    rng = random.Random(seed)
    nthr = nctas * tpc
    ncomp = nthr + 2 * nctas            # threads, then one table and one exchange copy engine per CTA
    vcs = [_VC(ncomp) for _ in range(nthr)]
    for t in range(nthr):
        vcs[t].v[t] = 1
    pc = [0] * nthr
    c_arr: dict[int, list] = {}
    c_next_arrive = [0] * nthr
    c_next_wait = [0] * nthr
    s_gen = [0] * nctas
    s_count = [0] * nctas
    s_vc = [_VC(ncomp) for _ in range(nctas)]
    s_waiting = [None] * nthr
    t_issued = [[] for _ in range(nctas)]
    t_done = [[] for _ in range(nctas)]
    t_next = [0] * nthr
    x_issued: dict[tuple, list] = {}      # (dst, phase) -> copies
    x_sent = [[0] * nctas for _ in range(nctas)]   # x_sent[src][dst]: copies src issued to dst
    x_next = [0] * nthr
    ce_count = [0] * (2 * nctas)
    accesses: dict = {}
    races = []

    def access(loc, kind, epoch, stage, vc, who):
        lst = accesses.setdefault(loc, [])
        for pk, pe, ps, pvc, pwho in lst:
            if pk == "r" and kind == "r":
                continue
            if (pe, ps) == (epoch, stage):
                continue
            if pvc.v[pwho] > vc.v[pwho]:
                races.append((loc, (pk, pe, ps, pwho), (kind, epoch, stage, who)))
        lst.append((kind, epoch, stage, vc.copy(), who))

    def engine(cta, which):
        idx = nthr + 2 * cta + which
        ce_count[2 * cta + which] += 1
        return idx, ce_count[2 * cta + which]

    def runnable(t):
        prog = programs[t]
        if pc[t] >= len(prog):
            return False
        op = prog[pc[t]]
        cta = t // tpc
        if op[0] == "cwait":
            arr = c_arr.get(c_next_wait[t])
            return arr is not None and arr[0] == nthr
        if op[0] == "sync":
            return s_waiting[t] is None
        if op[0] == "twait":
            return len(t_issued[cta]) > t_next[t]
        if op[0] == "xwait":
            return len(x_issued.get((cta, x_next[t]), [])) >= op[1]
        return True

    while True:
        ready = [t for t in range(nthr) if runnable(t)]
        if not ready:
            if all(pc[t] >= len(programs[t]) for t in range(nthr)):
                # accesses to a CTA's memory from outside it must happen before that CTA exits
                for loc, lst in accesses.items():
                    owner = loc[1]
                    for k_, e_, s_, avc, who in lst:
                        if who < nthr and who // tpc == owner:
                            continue
                        if not any(avc.v[who] <= vcs[u].v[who] for u in range(owner * tpc, (owner + 1) * tpc)):
                            races.append((loc, (k_, e_, s_, who), "after the owner CTA exited"))
                return {"deadlock": None, "races": races}
            stuck = {t: programs[t][pc[t]] for t in range(nthr) if pc[t] < len(programs[t])}
            return {"deadlock": stuck, "races": races}
        t = rng.choice(ready)
        cta = t // tpc
        op = programs[t][pc[t]]
        vc = vcs[t]
        kind = op[0]
        if kind == "carrive":
            ph = c_next_arrive[t]
            if c_next_arrive[t] != c_next_wait[t]:
                raise AssertionError(f"thread {t}: two cluster arrives without a wait")
            arr = c_arr.setdefault(ph, [0, _VC(ncomp)])
            arr[0] += 1
            arr[1].join(vc)
            c_next_arrive[t] += 1
            pc[t] += 1
        elif kind == "cwait":
            ph = c_next_wait[t]
            if c_next_arrive[t] <= ph:
                raise AssertionError(f"thread {t}: cluster wait before its arrive")
            vc.join(c_arr[ph][1])
            c_next_wait[t] += 1
            pc[t] += 1
        elif kind == "sync":
            s_vc[cta].join(vc)
            s_count[cta] += 1
            s_waiting[t] = s_gen[cta]
            if s_count[cta] == tpc:
                gen_vc = s_vc[cta]
                s_vc[cta] = _VC(ncomp)
                s_count[cta] = 0
                s_gen[cta] += 1
                for u in range(cta * tpc, (cta + 1) * tpc):
                    vcs[u].join(gen_vc)
                    s_waiting[u] = None
                    pc[u] += 1
        elif kind == "tma":
            t_issued[cta].append((op[1], vc.copy()))
            pc[t] += 1
        elif kind == "twait":
            k = t_next[t]
            while len(t_done[cta]) <= k:
                tag, ivc = t_issued[cta][len(t_done[cta])]
                idx, n = engine(cta, 0)
                cvc = ivc.copy()
                cvc.v[idx] = n
                access(("Tb", cta), "w", ("slab", tag), "tma", cvc, idx)
                t_done[cta].append(cvc)
            vc.join(t_done[cta][k])
            t_next[t] += 1
            pc[t] += 1
        elif kind == "bulk":
            _, dst, src_loc, dst_loc, epoch = op
            ph = x_sent[cta][dst]
            x_sent[cta][dst] += 1
            x_issued.setdefault((dst, ph), []).append([vc.copy(), src_loc, dst_loc, epoch, None])
            pc[t] += 1
        elif kind == "xwait":
            ph = x_next[t]
            for cp in x_issued[(cta, ph)]:
                if cp[4] is None:
                    ivc, src_loc, dst_loc, epoch, _ = cp
                    idx, n = engine(cta, 1)
                    cvc = ivc.copy()
                    cvc.v[idx] = n
                    access(src_loc, "r", epoch, "bulk", cvc, idx)
                    access(dst_loc, "w", epoch, "bulk", cvc, idx)
                    cp[4] = cvc
                vc.join(cp[4])
            x_next[t] += 1
            pc[t] += 1
        elif kind == "acc":
            _, loc, k_, epoch, stage = op
            access(loc, k_, epoch, stage, vc, t)
            pc[t] += 1
        else:
            raise ValueError(op)
        vc.v[t] += 1
