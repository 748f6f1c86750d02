"""Host logic of bench.py that needs no GPU: the nvidia-smi clock record (median and maximum SM
clock, throttle reasons that reject a run), the algorithmic work and traffic figures the roofline
divides by, and the time-step rule of the shock tube."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProc:
    def __init__(self, lines, out):
        out.write("".join(lines))
        out.flush()

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clocks(monkeypatch, tmp_path, lines):
    monkeypatch.setattr(bench.subprocess, "Popen", lambda cmd, stdout, stderr: _FakeProc(lines, stdout))
    return bench.Clocks(0, str(tmp_path / "clocks.csv")).stop()


def _row(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return f"0, {sm}, {smax}, 900.5, 0x0, {hw}, {hwt}, {swt}, {pcap}\n"


def test_clock_record_median_and_reasons(monkeypatch, tmp_path):
    lines = [_row(2070, 2070), _row(2055, 2070, pcap="Active"), _row(1980, 2070), "garbage line\n",
             "0, [N/A], 2070, 1, 0, Not Active, Not Active, Not Active, Not Active\n"]
    rec = _clocks(monkeypatch, tmp_path, lines)
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 3


def test_clock_record_flags_slowdowns(monkeypatch, tmp_path):
    lines = [_row(1500, 2070, hw="Active"), _row(1600, 2070, hwt="Active", swt="Active")]
    rec = _clocks(monkeypatch, tmp_path, lines)
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_samples_or_tool(monkeypatch, tmp_path):
    assert _clocks(monkeypatch, tmp_path, [])["reasons"] == ["no samples"]

    def missing(*a, **k):
        raise FileNotFoundError("nvidia-smi")

    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    rec = bench.Clocks(0, str(tmp_path / "c2.csv")).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_work_figures():
    # (2M+2) real 3-D transforms of 2.5 N_v log2 N_v flops plus (4M+20) N_v pointwise, n = 32, M = 32
    nv = 32 ** 3
    assert bench.flops_per_cell() == pytest.approx(66 * 2.5 * nv * 15 + 148 * nv, rel=1e-15)
    assert bench.flops_per_cell() * bench.NCELLS == pytest.approx(2.816424804352e12, rel=1e-12)
    # split-BF16 path: 34 transforms x 3 passes x 8 tiles x 12 MMAs of 128 x 64 x 16
    assert bench.tc_issued_flops_per_cell() == 34 * 3 * 8 * 12 * (2 * 128 * 64 * 16)
    assert bench.PTS == 32 ** 3 * 32 ** 3


def test_traffic_scales_with_cells():
    for k, per_cell in bench.DRAM_BYTES_PER_CELL.items():
        assert bench.traffic(k) == pytest.approx(per_cell * bench.NCELLS)
    # the FP32 collision reads f and writes Q once: 8 bytes per point per launch, less the writes of a
    # capture's last cells still in L2 when it ends (7 % on 2048 cells)
    assert bench.DRAM_BYTES_PER_CELL["collide_f32"] == pytest.approx(8 * 32 ** 3, rel=0.1)
    assert bench.DRAM_BYTES_PER_CELL["bgk_f32"] == pytest.approx(8 * 32 ** 3, rel=0.1)
    assert bench.traffic("no such kernel") is None


def test_time_step_rule():
    dx, vmax = 1.0 / 32, (16 - 0.5) * (20.0 / 32)
    assert bench.dt_rule() == min(dx / vmax, 0.5 * 0.01 / 5.0)
    assert np.isclose(bench.dt_rule(), 1e-3)
