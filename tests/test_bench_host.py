"""Host-side logic of bench.py, no GPU: the algorithmic half-pair count, the
roofline arithmetic of the two pair kernels, and the DRAM-traffic record that
is keyed to the pair kernels' source (a kernel edited after its ncu capture
must report traffic null)."""
import json
import math
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Sys:
    def __init__(self, n):
        self.n = n


def test_half_pairs_are_the_cutoff_sphere_count():
    # N/2 times the atoms in a sphere of radius r_c at the box's density
    hp = bench.half_pairs_of([_Sys(1000), _Sys(500)],
                             [{"box": (30.0, 30.0, 30.0)}, {"box": (20.0, 25.0, 40.0)}], rc=10.0)
    sphere = 4.0 / 3.0 * math.pi * 1000.0
    want = 0.5 * 1000 * sphere * (1000 / 27000.0) + 0.5 * 500 * sphere * (500 / 20000.0)
    assert hp == pytest.approx(want, rel=1e-14)


def test_fp32_pair_roofline_is_bound_by_the_fp32_pipe():
    # 67 FP32 operations per half-pair on 128 lanes outweigh 11 MUFU results on 32
    hp, ms, clk = 6.3e6, 0.095, 2070e6
    rec = bench.pair_roofline(hp, ms, 1, clk)
    peak = 152 * 128 * clk / 1e12
    achieved = hp * 67 / (ms * 1e-3) / 1e12
    assert rec["unit"] == "Top/s (FP32 pipe)"
    assert rec["peak"] == pytest.approx(peak, rel=1e-12)
    assert rec["achieved"] == pytest.approx(achieved, rel=1e-12)
    assert rec["frac"] == pytest.approx(achieved / peak, rel=1e-12)
    assert rec["bound"] == "alu" and rec["units_per_launch"] == hp


def test_fp64_pair_roofline_counts_the_fp64_pipe():
    hp, ms, clk = 6.25e6, 1.38, 2070e6
    rec = bench.pair_roofline(hp, ms, 0, clk)
    peak = 152 * 2 * clk / 1e12
    assert rec["kernel"] == "k_pair_f64"
    assert rec["frac"] == pytest.approx(hp * 79 / (ms * 1e-3) / 1e12 / peak, rel=1e-12)


def test_no_launch_time_gives_no_roofline():
    assert bench.pair_roofline(6.3e6, None, 1, 2070e6) is None


def test_traffic_record_matches_the_current_pair_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "pair_kernel.json")))
    assert bench.pair_traffic("water", 1) == rec["dram_bytes_per_launch"]["water_fp32"]
    assert bench.pair_traffic("water", 0) == rec["dram_bytes_per_launch"]["water_fp64"]


def test_traffic_is_null_once_the_pair_source_changes(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "pair_kernel.json"), tmp_path / "profiles")
    src = tmp_path / "paper_2602_23582_gb300" / "csrc"
    src.mkdir(parents=True)
    text = open(os.path.join(ROOT, "paper_2602_23582_gb300", "csrc", "k_pair.cu")).read()
    (src / "k_pair.cu").write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.pair_traffic("water", 1) is not None
    (src / "k_pair.cu").write_text(text + "\n// edited\n")
    assert bench.pair_traffic("water", 1) is None
