"""Host-side parts of bench.py, without a GPU: the clock-sample summary that
decides whether a run is kept, the kernel-class shares, and the JSON line
of the reference arm (the oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_reads_median_and_reasons():
    c = bench.ClockSampler(0)
    # index, sm, max sm, power, active mask, hw, hw thermal, sw thermal, sw power cap
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    c.lines.append("0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["reasons"] == []


def test_class_shares_sum_to_one_over_launched_classes():
    prof = {"combine": (60.0, 10, 1.0, 1.0), "gram": (30.0, 5, 1.0, 1.0),
            "cg": (10.0, 2, 0.0, 0.0), "unused": (0.0, 0, 0.0, 0.0)}
    sh = bench.class_shares(prof)
    assert set(sh) == {"combine", "gram", "cg"}
    assert sh["combine"] == 0.6 and abs(sum(sh.values()) - 1.0) < 1e-12


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "solves/s"
    for key in ("metric", "value", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == bench.WORKLOAD
    # a step is one timed oracle iteration: steps x ms_per_step is the timed
    # work, and the extrapolated solve is reported separately
    cfg = line["config"]
    assert line["ms_per_step"] == pytest.approx(1e3 * cfg["oracle_seconds_per_iteration"])
    assert cfg["extrapolated_solve_seconds"] == pytest.approx(1.0 / line["value"])
    st = cb["single_thread"]
    assert st["seconds_per_iteration"] > 0 and st["value"] > 0


def test_roofline_of_the_dominant_class():
    peaks = {"sms": 152, "fp32_tflops": 78.0, "fp64_tflops": 1.1}
    clocks = {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0}
    # an FP32 contraction class dominates: FMA bound against unit counts x clock
    prof = {"combine": (50.0, 100, 2.0e12, 1.0e10), "hamiltonian": (20.0, 40, 1e9, 4.0e10)}
    r = bench.roofline(prof, clocks, peaks)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    assert r["achieved"] == pytest.approx(2.0e12 / 0.05 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_of_probe"] == pytest.approx(r["achieved"] / 78.0)
    # the class's DRAM traffic per launch comes from an ncu capture of its kernel
    assert r["traffic"] == bench.CLASS_TRAFFIC["combine"][0] and r["traffic_source"]
    # a stencil class dominates: HBM bound in GB/s
    prof = {"combine": (5.0, 10, 2.0e11, 1.0e9), "hamiltonian": (20.0, 40, 1e9, 4.0e10)}
    r = bench.roofline(prof, clocks, peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(4.0e10 / 0.02 / 1e9)
    assert r["traffic"] is None
