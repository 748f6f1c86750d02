"""Benchmark: phase-space points per second of one full FKS step (transport +
fast spectral collision + projected Euler update) on the 3D/3D hard-sphere
shock tube, 32^3 cells x 32^3 velocities, FP32, M = 32 directions.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space pts/s per step (N_v=32^3), learned+BF16 vs FP64 spectral @1e-3"
NX, NV, LBOX, KN, A1, A2 = 32, 32, 10.0, 0.01, 4, 8
M = A1 * A2
GRID = (NX, NX, NX)
NCELLS = NX ** 3
PTS = NCELLS * NV ** 3
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12     # SMs x FP64 FMA lanes x FMA x max SM clock (1.26 TFLOP/s)


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0   # fallback figure for a GB300


HBM_PEAK_GBS = _hbm_peak()


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback"


BF16_PEAK_TFLOPS, BF16_PEAK_KIND = _bf16_peak()


# DRAM bytes per cell of one launch (dram__bytes_read.sum + dram__bytes_write.sum of one
# ncu capture on the 16x16x8 = 2048-cell shock tube, divided by 2048; traffic grows with
# the cells of a launch).  Valid for the kernels as profiled; None once a kernel changes.
DRAM_BYTES_PER_CELL = {
    "collide_f32": (275447296 + 222745088) / 2048,   # collide_kernel<float, 32, 8>
    "bgk_f32": (268507392 + 215125504) / 2048,       # bgk_cluster_kernel<float, 32, 4> (f* read once)
    "collide_tc": (634375680 + 1517931008) / 2048,   # collide_tc_kernel<32> (scratch written back from L2)
}


def traffic(kernel):
    b = DRAM_BYTES_PER_CELL.get(kernel)
    return None if b is None else b * NCELLS


def tc_issued_flops_per_cell(n=NV, m=M):
    """Tensor-core flops the split-BF16 path issues per cell: (M + 2) complex 3-D
    transforms x 3 passes x n^2/128 tiles x (2n/16 k-steps x 3 split products)
    MMAs of 128 x 2n x 16."""
    k = 2 * n
    return (m + 2) * 3 * (n * n // 128) * (k // 16) * 3 * (2 * 128 * k * 16)


def flops_per_cell(n=NV, m=M):
    """Algorithmic flops of the operator per cell: (2M+2) real 3-D transforms
    at 2.5 N_v log2 N_v each, plus (4M+20) N_v pointwise."""
    nv = n ** 3
    return (2 * m + 2) * 2.5 * nv * np.log2(nv) + (4 * m + 20) * nv


def dt_rule():
    """dt = min(dx / max|v|, 0.5 Kn / nu_max) with nu_max ~ 5 for rho = T = 1."""
    dx = 1.0 / NX
    vmax = (NV / 2 - 0.5) * (2 * LBOX / NV)
    return min(dx / vmax, 0.5 * KN / 5.0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """Maximum of a per-rank scalar (the slowest rank sets the time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(sample_cells: int = 16, fp32_input=None) -> dict:
    """The oracle as it stands, on `sample_cells` cells of the workload, on
    this host's cores (OpenMP over cells)."""
    import oracle
    from paper_1701_01608_gb300 import inputs as I
    oracle.build()
    t0 = time.perf_counter()
    tab = oracle.tables(NV, LBOX, 0, 0.25, A1, A2, 0)
    t_tab = time.perf_counter() - t0
    states, which = I.shock_tube_states(NV, LBOX, NX)
    rng = np.random.Generator(np.random.PCG64(12345))
    cells = rng.choice(NCELLS, size=sample_cells, replace=False)
    f = np.stack([states[which[c // (NX * NX)]] for c in cells])
    t0 = time.perf_counter()
    Q = oracle.collide(f, tab, kn=KN, project=True)
    dt = dt_rule()
    _ = f + dt * Q
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": sample_cells * NV ** 3 / el, "unit": "pts/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
            "sample": f"{sample_cells} seeded cells of the 32^3x32^3 shock tube, collision + Euler "
                      f"(transport gather is a copy, excluded); tables {t_tab:.1f}s excluded",
            "seconds": el}


def learned_path(torch, fks, dev, args, sample=1216, threshold=1e-3):
    """Learned surrogate collision (BF16 conv net, calibrated indicator, cells over the
    threshold routed to the FP32 spectral operator) against the FP32 spectral collision
    and the FP64 spectral operator, on a sample of non-equilibrium cells of the
    workload's velocity grid (shock-tube cells after a few steps, two-stream cells)."""
    from paper_1701_01608_gb300 import surrogate as S
    t0 = time.perf_counter()
    ftr = torch.cat([S.shock_tube_cells(torch, NV, LBOX, nx=32, ny=2, nz=2, steps=(0, 4, 8, 16), seed=0),
                     S.two_stream_cells(torch, 128, NV, LBOX, seed=1)])
    Qtr = S.labels(torch, ftr, NV, LBOX, kn=1.0)
    sur = S.train(torch, ftr, Qtr, epochs=8, batch=8, lr=2e-3, n=NV, L=LBOX, holdout=0.2)
    train_s = time.perf_counter() - t0
    del ftr, Qtr
    f = torch.cat([S.shock_tube_cells(torch, NV, LBOX, nx=32, ny=8, nz=4, steps=(6,), seed=5)[:sample - 192],
                   S.two_stream_cells(torch, 192, NV, LBOX, seed=9)]).contiguous()
    nc = f.shape[0]
    c32 = fks.Context(fks.Config(ncell=(nc, 1, 1), n=NV, L=LBOX, kn=KN, A1=A1, A2=A2, precision=fks.FKS_FP32))
    c64 = fks.Context(fks.Config(ncell=(nc, 1, 1), n=NV, L=LBOX, kn=KN, A1=A1, A2=A2, precision=fks.FKS_FP64))
    Q64 = torch.empty(f.shape, dtype=torch.float64, device=dev)
    c64.collide(f.double(), Q64)
    Qs = torch.empty_like(f)
    Ql = torch.empty_like(f)

    def timed(fn, reps=5):
        """median over reps of the per-call device time (one call includes a host sync)"""
        fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        ev[0].record()
        for i in range(reps):
            fn()
            ev[i + 1].record()
        torch.cuda.synchronize()
        return float(np.median([ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]))

    t_spec = timed(lambda: c32.collide(f, Qs))
    routed = [0]
    t_learn = timed(lambda: routed.__setitem__(0, c32.surrogate_collide(sur.net, f, Ql, sur.out_scale,
                                                                        sur.ind_scale, threshold)))

    def err(Q):
        d = (Q.double() - Q64).flatten(1).norm(dim=1) / Q64.flatten(1).norm(dim=1)
        return float(d.max().item()), float(d.median().item())

    # the learned + split-BF16 path: routed cells recomputed on the tensor cores
    ctc = fks.Context(fks.Config(ncell=(nc, 1, 1), n=NV, L=LBOX, kn=KN, A1=A1, A2=A2, precision=fks.FKS_BF16X3))
    Qt, Qlt = torch.empty_like(f), torch.empty_like(f)
    t_tc = timed(lambda: ctc.collide(f, Qt))
    routed_t = [0]
    t_learn_tc = timed(lambda: routed_t.__setitem__(0, ctc.surrogate_collide(sur.net, f, Qlt, sur.out_scale,
                                                                              sur.ind_scale, threshold)))
    elt, mlt = err(Qlt)
    del ctc
    el, ml = err(Ql)
    es, ms = err(Qs)
    pts = nc * NV ** 3
    return {"value": pts / (t_learn / 1e3), "unit": "pts/s", "ms": t_learn, "cells": nc,
            "routed_fraction": routed[0] / nc, "threshold": threshold,
            "err_vs_fp64": {"max": el, "median": ml},
            "spectral_fp32_collide": {"value": pts / (t_spec / 1e3), "ms": t_spec, "err_vs_fp64": {"max": es, "median": ms}},
            "speedup_vs_spectral_fp32": t_spec / t_learn,
            "learned_bf16x3": {"value": pts / (t_learn_tc / 1e3), "ms": t_learn_tc, "routed_fraction": routed_t[0] / nc,
                               "err_vs_fp64": {"max": elt, "median": mlt},
                               "spectral_bf16x3_collide_ms": t_tc,
                               "note": "routed cells recomputed by the split-BF16 tensor-core operator"},
            "err_note": "relative L2 of Q against the FP64 operator on this sample, which includes nearly "
                        "Maxwellian shock-tube cells: there ||L|| / ||Q|| is large and the error is bounded on the "
                        "loss scale (FP32 2.5e-7 ||L||, split BF16 2.5e-5 ||L||); far from equilibrium see "
                        "bf16x3_tensor_core.err_vs_fp64",
            "train_seconds": train_s, "train_loss_last": sur.train_loss[-1], "calibration": sur.calib,
            "note": "collision operator only (the part the surrogate replaces), same sample for both paths; "
                    "net: 6 x conv3d 3^3, 32 ch, BF16 weights and activations, FP32 accumulation; inference on "
                    "the tensor cores (tcgen05 implicit GEMM), training on CUDA cores"}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle  # noqa: F401
    from paper_1701_01608_gb300 import inputs as I
    import oracle as O
    O.build()
    tab = O.tables(NV, LBOX, 0, 0.25, A1, A2, 0)
    states, which = I.shock_tube_states(NV, LBOX, NX)
    sample = int(os.environ.get("FKS_REF_SAMPLE", "256"))
    rng = np.random.Generator(np.random.PCG64(777))
    times = []
    for it in range(args.warmup + args.steps):
        cells = rng.choice(NCELLS, size=sample, replace=False)
        f = np.stack([states[which[c // (NX * NX)]] for c in cells])
        t0 = time.perf_counter()
        Q = O.collide(f, tab, kn=KN, project=True)
        _ = f + dt_rule() * Q
        el = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(el)
    sec = float(np.mean(times))
    val = sample * NV ** 3 / sec
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pts/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "hs_shocktube_32x32x32c_32v (sampled cells)", "cells_per_step": sample,
                      "n_v": NV ** 3, "M": M, "note": "CPU oracle (plain FP64 C, OpenMP over cells)"},
           "cpu_baseline": {"value": val, "unit": "pts/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                            "sample": f"{sample} seeded cells per step"},
           "e2e": {"value": val, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def build_state(torch, dtype, dev):
    from paper_1701_01608_gb300 import inputs as I
    states, which = I.shock_tube_states(NV, LBOX, GRID[0])
    st = torch.from_numpy(states).to(device=dev, dtype=dtype)
    idx = torch.from_numpy(np.repeat(which, GRID[1] * GRID[2])).to(dev)
    return st.index_select(0, idx).contiguous()


def time_steps(torch, ctx, f0, steps, warmup, dt, ws):
    fa = f0.clone()
    fb = torch.empty_like(fa)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.step(fa, fb, dt)
        fa, fb = fb, fa
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    launches0 = ctx.launches
    ev[0].record(stream)
    for i in range(steps):
        ctx.step(fa, fb, dt)
        fa, fb = fb, fa
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = ev[0].elapsed_time(ev[steps])
    bits = ctx.check()
    return total_ms, per, ctx.launches - launches0, bits, fa


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-bgk", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-tc", action="store_true")
    ap.add_argument("--no-varb", action="store_true")
    ap.add_argument("--no-vhs", action="store_true")
    ap.add_argument("--no-strang", action="store_true")
    ap.add_argument("--clocks-log", default=None, help="keep the raw nvidia-smi clock samples of the timed "
                                                        "region in this CSV file")
    ap.add_argument("--cpu-sample", type=int, default=int(os.environ.get("FKS_CPU_SAMPLE", "1024")))
    ap.add_argument("--grid", default=None, help="nx,ny,nz spatial cells (default 32,32,32); smaller grids "
                    "are for profiling runs, not bench lines")
    args = ap.parse_args()
    global GRID, NCELLS, PTS
    if args.grid:
        GRID = tuple(int(v) for v in args.grid.split(","))
        NCELLS = GRID[0] * GRID[1] * GRID[2]
        PTS = NCELLS * NV ** 3
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = dist_setup()
    cpu = None
    if rank == 0 and ws == 1 and args.cpu_sample > 0:
        # the oracle runs before any CUDA call (OpenMP, no fork after CUDA init)
        cpu = cpu_baseline(args.cpu_sample)
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1701_01608_gb300 import fks
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    dt = dt_rule()
    cfg = fks.Config(ncell=GRID, bc=(1, 0, 0), n=NV, L=LBOX, kernel=0, C=0.25, kn=KN,
                     A1=A1, A2=A2, precision=fks.FKS_FP32)
    ctx = fks.Context(cfg)
    f0 = build_state(torch, torch.float32, dev)
    # measured FMA throughput of the FP32 and FP64 pipes (a second denominator beside the derived one)
    alu32 = fks.alu_peak(fks.FKS_FP32)
    alu64 = fks.alu_peak(fks.FKS_FP64)

    clk = Clocks(torch.cuda.current_device(),
                 args.clocks_log or os.path.join(tempfile.gettempdir(), f"fks_clocks_{os.getpid()}_{rank}.csv"))
    total_ms, per, launches, bits, _ = time_steps(torch, ctx, f0, args.steps, args.warmup, dt, ws)
    clocks = clk.stop()
    total_ms = max_over_ranks(total_ms, ws)
    sec = total_ms / 1e3
    value = ws * PTS * args.steps / sec
    step_ms = float(np.mean(per))
    flops_launch = flops_per_cell() * NCELLS
    achieved = flops_launch / (step_ms / 1e3) / 1e12

    # stage timers (CUDA events, each stage alone; the step fuses transport, collision,
    # projection and the Euler update into one kernel)
    stages = None
    if ws == 1:
        tmp = torch.empty_like(f0)
        U = torch.empty((NCELLS, 5), dtype=torch.float64, device=dev)

        def ev_ms(fn, reps=2):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        stages = {"transport_ms": ev_ms(lambda: ctx.transport(f0, tmp, dt)),
                  "moments_ms": ev_ms(lambda: ctx.moments(f0, U)),
                  "collide_ms": ev_ms(lambda: ctx.collide(f0, tmp)),
                  "step_ms": step_ms,
                  "note": "FP32; transport = offsets + gather kernel (2 x 4 B per point), moments = compensated "
                          "FP32 sums (FP64-equivalent), 4 B per point"}
        del tmp, U

    e2e = None
    if not args.no_e2e:
        # public API with host buffers: H2D of the step's input, the step, D2H of the result
        host_in = torch.empty(f0.shape, dtype=torch.float32, pin_memory=True)
        host_in.copy_(f0)
        host_out = torch.empty_like(host_in, pin_memory=True)
        e2e_steps = max(1, min(args.steps, 5))
        # fks_step_host: the library copies the step's input in, steps and copies the result out,
        # pipelined over x-slab chunks (every step: H2D of the whole state, the step, D2H)
        ctx.step_host(host_in, host_out, dt)
        torch.cuda.synchronize()
        barrier(ws)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
        evs[0].record()
        for i in range(e2e_steps):
            ctx.step_host(host_in, host_out, dt)
            evs[i + 1].record()
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(evs[0].elapsed_time(evs[e2e_steps]), ws)
        e2e_each = [round(evs[i].elapsed_time(evs[i + 1]), 2) for i in range(e2e_steps)]
        nbytes = f0.numel() * 4
        # plain copy rates between the pinned host arrays and the device (one full-state copy each
        # way), to read the e2e line against
        dtmp = torch.empty_like(f0)
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record()
        dtmp.copy_(host_in, non_blocking=True)
        c1.record()
        host_out.copy_(dtmp, non_blocking=True)
        c2.record()
        torch.cuda.synchronize()
        copy_gbs = {"h2d": nbytes / (c0.elapsed_time(c1) / 1e3) / 1e9,
                    "d2h": nbytes / (c1.elapsed_time(c2) / 1e3) / 1e9}
        del dtmp
        e2e = {"value": ws * PTS * e2e_steps / (e2e_ms / 1e3), "unit": "pts/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e2e_steps, "ms_each": e2e_each,
               "ms_median": float(np.median(e2e_each)), "copy_gbs": copy_gbs,
               "api": "fks_step_host (pinned host arrays; copies overlapped with the step over 8 x-slab chunks)"}
        del host_in, host_out

    # BGK relaxation step on the same workload: HBM bound (8 B per point)
    bgk = None
    if not args.no_bgk:
        cfgb = fks.Config(ncell=GRID, bc=(1, 0, 0), n=NV, L=LBOX, kernel=fks.BGK, kn=KN, precision=fks.FKS_FP32)
        ctxb = fks.Context(cfgb)
        tb, perb, _, _, _ = time_steps(torch, ctxb, f0, args.steps, args.warmup, dt, ws)
        tb = max_over_ranks(tb, ws)
        bms = float(np.mean(perb))
        gbs = 8.0 * PTS / (bms / 1e3) / 1e9
        bgk = {"value": ws * PTS * args.steps / (tb / 1e3), "unit": "pts/s", "ms_per_step": tb / args.steps,
               "roofline": {"bound": "hbm", "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                            "frac": gbs / HBM_PEAK_GBS, "traffic": traffic("bgk_f32"),
                            "algorithmic_bytes_per_launch": 8.0 * PTS,
                            "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
               "note": "BGK relaxation (Sec. 2) with the fused transport gather, FP32"}
        # the stiff (exponential) BGK step at Kn = 1e-6, nu dt ~ 1e3, where the Euler step diverges
        ctxe = fks.Context(fks.Config(ncell=GRID, bc=(1, 0, 0), n=NV, L=LBOX, kernel=fks.BGK, kn=1e-6,
                                      precision=fks.FKS_FP32))
        fa, fb = f0.clone(), torch.empty_like(f0)
        for _ in range(max(1, min(args.warmup, 3))):
            ctxe.step_exp(fa, fb, dt)
            fa, fb = fb, fa
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            ctxe.step_exp(fa, fb, dt)
            fa, fb = fb, fa
        e1.record()
        torch.cuda.synchronize()
        bgk["stiff_exp_step"] = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "knudsen": 1e-6,
                                 "health_bits": ctxe.check(),
                                 "note": "fks_step_exp: transport + exact BGK relaxation over dt (stable at any nu dt)"}
        del ctxb, ctxe, fa, fb

    # the same step with every DFT on the tensor cores (split BF16)
    tcp = None
    if not args.no_tc:
        cfgt = fks.Config(ncell=GRID, bc=(1, 0, 0), n=NV, L=LBOX, kernel=0, C=0.25, kn=KN,
                          A1=A1, A2=A2, precision=fks.FKS_BF16X3)
        ctxt = fks.Context(cfgt)
        tt, pert, launches_t, bits_t, _ = time_steps(torch, ctxt, f0, args.steps, args.warmup, dt, ws)
        tt = max_over_ranks(tt, ws)
        tms = float(np.mean(pert))
        issued = tc_issued_flops_per_cell() * NCELLS
        tfl = issued / (tms / 1e3) / 1e12
        tcp = {"value": ws * PTS * args.steps / (tt / 1e3), "unit": "pts/s", "ms_per_step": tt / args.steps,
               "roofline": {"bound": "tensor", "achieved": tfl, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tfl / BF16_PEAK_TFLOPS, "traffic": traffic("collide_tc"),
                            "issued_flops_per_launch": issued,
                            "peak_note": "bf16_tflops_sustained of MEASURED_PEAKS.json (%s); issued split-BF16 "
                                         "MMA flops (3 products per DFT)" % BF16_PEAK_KIND},
               "algorithmic_tflops": flops_launch / (tms / 1e3) / 1e12,
               "gpu_launches": launches_t, "health_bits": bits_t,
               "note": "fks_step on an FKS_BF16X3 context: offsets + one tcgen05 kernel per step (split-BF16 "
                       "DFT passes, FP32 between passes, FP64 moment sums)"}
        if ws == 1:
            # error of the collision operator against the FP64 GPU operator on cells far from
            # equilibrium (the initial shock-tube cells are Maxwellians, Q ~ 0 there)
            from paper_1701_01608_gb300 import inputs as I
            fs = torch.from_numpy(I.two_stream((64, 1, 1), NV, LBOX, seed=77, noise=0.05).astype(np.float32)).to(dev)
            errs = {}
            qref = torch.empty(fs.shape, dtype=torch.float64, device=dev)
            fks.Context(fks.Config(ncell=(64, 1, 1), n=NV, L=LBOX, kernel=0, C=0.25, kn=KN, A1=A1, A2=A2,
                                   precision=fks.FKS_FP64)).collide(fs.double(), qref)
            for name, prec in (("bf16x3", fks.FKS_BF16X3), ("fp32", fks.FKS_FP32)):
                q = torch.empty_like(fs)
                fks.Context(fks.Config(ncell=(64, 1, 1), n=NV, L=LBOX, kernel=0, C=0.25, kn=KN, A1=A1, A2=A2,
                                       precision=prec)).collide(fs, q)
                d = ((q.double() - qref).flatten(1).norm(dim=1) / qref.flatten(1).norm(dim=1)).cpu().numpy()
                errs[name] = {"max": float(d.max()), "median": float(np.median(d))}
            tcp["err_vs_fp64"] = errs
            tcp["err_sample"] = "64 seeded two-stream cells (5 % noise) on the workload's velocity grid, relative L2 of Q"
        del ctxt

    # variant B (de-aliased, 2n transforms) in the paper's own setting: 16^3 modes with 32^3 transforms
    varb = None
    if not args.no_varb and ws == 1:
        from paper_1701_01608_gb300 import inputs as I
        nb = 16
        states, which = I.shock_tube_states(nb, LBOX, GRID[0])
        sb = torch.from_numpy(states).float().to(dev)
        fb0 = sb.index_select(0, torch.from_numpy(np.repeat(which, GRID[1] * GRID[2])).to(dev)).contiguous()
        res = {}
        for name, dealias in (("variant_b", True), ("variant_a", False)):
            cb = fks.Context(fks.Config(ncell=GRID, bc=(1, 0, 0), n=nb, L=LBOX, kernel=0, C=0.25, kn=KN, A1=A1, A2=A2,
                                        precision=fks.FKS_FP32, dealias=dealias))
            tb_, perb_, lb_, bitsb_, _ = time_steps(torch, cb, fb0, args.steps, args.warmup, dt, ws)
            res[name] = {"ms_per_step": tb_ / args.steps, "value": NCELLS * nb ** 3 * args.steps / (tb_ / 1e3),
                         "gpu_launches": lb_, "health_bits": bitsb_}
            del cb
        # error of FP32 variant B against FP64 variant B on far-from-equilibrium cells
        fs = torch.from_numpy(I.two_stream((64, 1, 1), nb, LBOX, seed=78, noise=0.05)).to(dev)
        q64 = torch.empty_like(fs)
        fks.Context(fks.Config(ncell=(64, 1, 1), n=nb, L=LBOX, kernel=0, C=0.25, kn=KN, A1=A1, A2=A2,
                               precision=fks.FKS_FP64, dealias=True)).collide(fs, q64)
        q32 = torch.empty_like(fs, dtype=torch.float32)
        fks.Context(fks.Config(ncell=(64, 1, 1), n=nb, L=LBOX, kernel=0, C=0.25, kn=KN, A1=A1, A2=A2,
                               precision=fks.FKS_FP32, dealias=True)).collide(fs.float(), q32)
        d = ((q32.double() - q64).flatten(1).norm(dim=1) / q64.flatten(1).norm(dim=1)).cpu().numpy()
        ms_b = res["variant_b"]["ms_per_step"]
        fl2 = flops_per_cell(2 * nb, M) * NCELLS
        varb = {"value": res["variant_b"]["value"], "unit": "pts/s (N_v = 16^3)", "ms_per_step": ms_b,
                "variant_a_same_grid": res["variant_a"],
                "roofline": {"bound": "alu", "achieved": fl2 / (ms_b / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "frac": fl2 / (ms_b / 1e3) / 1e12 / FP32_PEAK_TFLOPS, "traffic": None,
                             "algorithmic_flops_per_launch": fl2,
                             "peak_note": "operator flops at the 2n = 32 grid; derived FP32 peak"},
                "gpu_launches": res["variant_b"]["gpu_launches"],
                "err_fp32_vs_fp64": {"max": float(d.max()), "median": float(np.median(d))},
                "note": "shock tube %dx%dx%d cells x 16^3 velocities, FP32, fks_step with fks_set_dealias: "
                        "interpolation to 32^3, the 32^3 collision without projection, truncation to "
                        "|k| <= 8 and projection (per 2048-cell chunk: 3 launches)" % GRID}
        del fb0, sb

    # variable hard spheres B = C|g|^alpha (non-separable Carleman kernel, expanded into
    # separable terms): Maxwell molecules, alpha = 0, on the same workload
    vhs = None
    if not args.no_vhs and ws == 1:
        from paper_1701_01608_gb300 import inputs as I
        alpha = 0.0
        _, S, trunc = fks.vhs_factor(alpha, 0.25, LBOX, NV, fks.FKS_FP32, 0, 0.0, 0.0)
        cv = fks.Context(fks.Config(ncell=GRID, bc=(1, 0, 0), n=NV, L=LBOX, kernel=fks.VHS, C=0.25, kn=KN,
                                    A1=A1, A2=A2, precision=fks.FKS_FP32, alpha=alpha))
        ks, kw = min(args.steps, 3), max(1, min(args.warmup, 3))
        tv, perv, lv, bitsv, _ = time_steps(torch, cv, f0, ks, kw, dt, ws)
        del cv
        msv = float(np.mean(perv))
        flv = flops_per_cell(NV, M * S) * NCELLS
        fs = torch.from_numpy(I.two_stream((8, 1, 1), NV, LBOX, seed=79, noise=0.05)).to(dev)
        q64 = torch.empty_like(fs)
        fks.Context(fks.Config(ncell=(8, 1, 1), n=NV, L=LBOX, kernel=fks.VHS, C=0.25, kn=KN, A1=A1, A2=A2,
                               precision=fks.FKS_FP64, alpha=alpha)).collide(fs, q64)
        q32 = torch.empty_like(fs, dtype=torch.float32)
        fks.Context(fks.Config(ncell=(8, 1, 1), n=NV, L=LBOX, kernel=fks.VHS, C=0.25, kn=KN, A1=A1, A2=A2,
                               precision=fks.FKS_FP32, alpha=alpha)).collide(fs.float(), q32)
        d = ((q32.double() - q64).flatten(1).norm(dim=1) / q64.flatten(1).norm(dim=1)).cpu().numpy()
        vhs = {"value": PTS * ks / (tv / 1e3), "unit": "pts/s", "ms_per_step": tv / ks, "steps": ks,
               "alpha": alpha, "terms": S, "truncation": trunc,
               "roofline": {"bound": "alu", "achieved": flv / (msv / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                            "unit": "TFLOP/s", "frac": flv / (msv / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                            "traffic": None, "algorithmic_flops_per_launch": flv,
                            "peak_note": "operator flops with M x terms table pairs; derived FP32 peak"},
               "gpu_launches": lv, "health_bits": bitsv,
               "err_fp32_vs_fp64": {"max": float(d.max()), "median": float(np.median(d))},
               "note": "fks_step, FKS_VHS alpha = 0 (Maxwell molecules, B = C): the radial factor of the "
                       "Carleman kernel 4C (|x|^2+|y|^2)^-1/2 expanded into %d separable terms, "
                       "%d table pairs per cell; same shock tube, FP32" % (S, M * S)}

    # second-order step (Strang splitting, Heun collision sub-step) on the same workload
    strang = None
    if not args.no_strang and ws == 1:
        cs = fks.Context(cfg)
        fa, fb, fw = f0.clone(), torch.empty_like(f0), torch.empty_like(f0)
        ks, kw = min(args.steps, 5), max(1, min(args.warmup, 3))
        for _ in range(kw):
            cs.step_strang(fa, fb, fw, dt)
            fa, fb = fb, fa
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = cs.launches
        e0.record()
        for _ in range(ks):
            cs.step_strang(fa, fb, fw, dt)
            fa, fb = fb, fa
        e1.record()
        torch.cuda.synchronize()
        tsr = e0.elapsed_time(e1)
        fls = 2 * flops_per_cell() * NCELLS / (tsr / ks / 1e3) / 1e12
        strang = {"value": PTS * ks / (tsr / 1e3), "unit": "pts/s", "ms_per_step": tsr / ks, "steps": ks,
                  "roofline": {"bound": "alu", "achieved": fls, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                               "frac": fls / FP32_PEAK_TFLOPS, "traffic": None,
                               "peak_note": "two operator evaluations per step; derived FP32 peak"},
                  "gpu_launches": cs.launches - l0, "health_bits": cs.check(),
                  "note": "fks_step_strang: T(dt/2), Heun collision (two projected operator evaluations), "
                          "T(dt/2); second order in dt; FP32, same workload and dt"}
        del cs, fa, fb, fw

    learned = None
    if not args.no_learned and ws == 1:
        learned = learned_path(torch, fks, dev, args)

    fp64 = None
    if not args.no_fp64 and ws == 1:
        cfg64 = fks.Config(ncell=GRID, bc=(1, 0, 0), n=NV, L=LBOX, kernel=0, C=0.25, kn=KN,
                           A1=A1, A2=A2, precision=fks.FKS_FP64)
        ctx64 = fks.Context(cfg64)
        f64 = build_state(torch, torch.float64, dev)
        t64, per64, _, _, _ = time_steps(torch, ctx64, f64, 1, 1, dt, ws)
        fl64 = flops_per_cell() * NCELLS / (t64 / 1e3) / 1e12
        fp64 = {"value": PTS / (t64 / 1e3), "unit": "pts/s", "ms_per_step": t64,
                "roofline": {"bound": "alu", "achieved": fl64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": fl64 / FP64_PEAK_TFLOPS, "traffic": None, "peak_measured": alu64,
                             "frac_of_measured": fl64 / alu64 if alu64 else None,
                             "peak_note": "derived FP64 CUDA-core peak: 152 SMs x 2 FP64 FMA lanes x 2 flop x "
                                          "2.07 GHz (GB300's reduced FP64 rate)"},
                "note": "same workload and step through the FP64 kernels (1 timed step after 1 warm-up)"}
        del f64, ctx64

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "hs_shocktube_%dx%dx%dc_32v" % GRID, "cells": NCELLS, "n_v": NV ** 3, "M": M,
                   "kernel": "hard spheres", "knudsen": KN, "bc": "specular x, periodic y z",
                   "dt": dt, "path": "fks_step: offsets + fused transport/collision/projection/Euler kernel",
                   "cluster_size": ctx.cluster_size, "l2": "inputs 4.3 GB > L2 (no flush needed)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic("collide_f32"),
                     "traffic_note": "dram bytes of one ncu capture on 2048 cells, scaled by the cells of a launch",
                     "algorithmic_flops_per_launch": flops_launch,
                     "peak_note": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)",
                     "peak_measured": alu32, "frac_of_measured": achieved / alu32 if alu32 else None,
                     "peak_measured_note": "FMA-chain kernel (fks_alu_peak), this run"},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
        "health_bits": bits,
        "stages": stages,
        "fp64_spectral": fp64,
        "bgk_step": bgk,
        "bf16x3_tensor_core": tcp,
        "variant_b_16v": varb,
        "vhs_maxwell": vhs,
        "strang_second_order": strang,
        "learned": learned,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
