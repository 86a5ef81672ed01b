"""Host-side logic of bench.py, on the CPU: the algorithmic-byte model of each kernel (the
roofline numerator), the DRAM-traffic scaling read from the committed ncu summary and keyed to
the step kernel's sources, the clock sampler's reading of nvidia-smi samples, the peak lookup
and the single-rank reduction."""
import json
import os

import pytest

import bench


def test_algorithmic_bytes_of_each_kernel():
    N, E, GC, MC = 1000, 10, 400, 441  # points, edges, cells, quads
    # fused step: points read and written (8 B each way), per-edge count in and out, group and
    # weight (16 B), the density once, the histogram written once
    assert bench.algorithmic_bytes("advect_resample", N, E, GC, 8, 4) == 16 * N + 16 * E + 4 * GC + 4 * GC
    assert bench.algorithmic_bytes("resample", N, E, GC, 8, 4) == 16 * N + 16 * E + 4 * GC
    assert bench.algorithmic_bytes("advect", N, E, GC, 8, 2) == 16 * N + 12 * E + 2 * GC
    assert bench.algorithmic_bytes("rowbox", N, E, GC, 8, 4) == GC * (4 + 8)
    assert bench.algorithmic_bytes("colbox", N, E, GC, 4, 4) == 2 * GC * 4
    # the mix reads the sums once and writes four densities per quad
    assert bench.algorithmic_bytes("mix_quads", N, E, GC, 8, 4, MC) == GC * 8 + 4 * MC * 4
    assert bench.algorithmic_bytes("mix_quads", N, E, GC, 8, 2) == GC * 8 + 4 * GC * 2
    assert bench.algorithmic_bytes("hist_clear", N, E, GC, 8, 4) == 0


def _profile_entry():
    path = os.path.join(bench.ROOT, "profiles", "k_step_lattice-1M-8groups.md")
    with open(path) as fh:
        text = fh.read()
    return json.loads(text.split("```json", 1)[1].split("```", 1)[0])["advect_resample"]


def test_measured_traffic_scales_the_captured_ratio(monkeypatch):
    ent = _profile_entry()
    assert ent["dram_bytes_per_launch"] > 0 and ent["algorithmic_bytes_per_launch"] > 0
    # keyed to the sources the capture was taken on
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: ent["source_hash"])
    got = bench.measured_traffic("advect_resample", 3.0e9)
    want = ent["dram_bytes_per_launch"] / ent["algorithmic_bytes_per_launch"] * 3.0e9
    assert got == pytest.approx(want, rel=1e-12)
    assert bench.measured_traffic("mix_quads", 3.0e9) is None  # no capture for that kernel


def test_measured_traffic_is_null_once_the_kernel_changed(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.measured_traffic("advect_resample", 3.0e9) is None


def test_source_hash_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    root = tmp_path
    csrc = root / "paper_1504_02687_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("k_points.cu", "density.cuh", "internal.cuh"):
        (csrc / f).write_text("int a = 1;\nint b = 2;\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_source_hash()
    (csrc / "density.cuh").write_text("// a new comment\nint a = 1;  // trailing\n\nint b = 2;\n")
    assert bench.kernel_source_hash() == h0
    (csrc / "density.cuh").write_text("int a = 1;\nint b = 3;\n")
    assert bench.kernel_source_hash() != h0


class _FakeSmi:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _sampler(lines):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = _FakeSmi("\n".join(lines) + "\n")
    return s


def test_clock_sampler_takes_the_loaded_samples_and_the_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "0, 2070, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1995, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1390.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c = _sampler(lines).stop()
    # the samples at or above the median power draw (1365 W): 1995 and 2010 MHz
    assert c["sm_mhz"] == pytest.approx(2002.5)
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert c["samples"] == 4


def test_clock_sampler_reports_a_hardware_slowdown():
    lines = ["0, 1500, 2070, 1300.0, 0x8, Active, Not Active, Not Active, Not Active"]
    c = _sampler(lines).stop()
    assert c["reasons"] == ["hw_slowdown"] and c["sm_mhz"] == 1500.0


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_and_single_rank_reduction():
    gbs, src = bench.peaks()
    assert gbs > 0 and src in ("measured", "fallback")
    assert bench.reduce_over_ranks(None, 4.25, 1.0e9) == (4.25, 1.0e9)
