"""The benchmark's host-side contract, checked without a GPU: the reference
arm (the oracle on the host cores) prints one JSON line with the required
keys, only rank 0 prints under a multi-rank launch, and the roofline
arithmetic divides the algorithmic work by the measured time."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(args, **env):
    e = dict(os.environ, **env)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=600)
    return r


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "GFlop/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFlop/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["backward_error"] <= 1e-13


def test_reference_arm_prints_nothing_on_other_ranks():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], RANK="1", WORLD_SIZE="2",
             LOCAL_RANK="1")
    assert r.returncode == 0 and not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_class_roofline_arithmetic():
    peaks = {"hbm_gbs": 5000.0, "bf16_tflops": 2000.0, "source": "of measured"}
    st = {"ms": 2.0, "launches": 7, "flops": 4e12, "bytes": 6e9}
    tc = bench.class_roofline("update_tc", st, "tf32", peaks)
    assert tc["bound"] == "hbm" and tc["unit"] == "GB/s"
    assert tc["achieved"] == pytest.approx(6e9 / 2e-3 / 1e9)
    assert tc["frac"] == pytest.approx(tc["achieved"] / 5000.0)
    assert tc["tensor"]["peak_tflops"] == pytest.approx(2000.0 * 1.1 / 2.25)
    assert tc["tensor"]["achieved_tflops"] == pytest.approx(4e12 / 2e-3 / 1e12)
    bf = bench.class_roofline("update_tc", st, "bf16", peaks)
    assert bf["tensor"]["peak_tflops"] == pytest.approx(2000.0)
    dg = bench.class_roofline("diag", st, "tf32", peaks)      # FP64 diagonal blocks in every mode
    assert dg["bound"] == "alu" and dg["peak"] == pytest.approx(bench.FP64_ALU_PEAK_GFLOPS)
    assert dg["achieved"] == pytest.approx(4e12 / 2e-3 / 1e9)
    up = bench.class_roofline("update", st, "tf32", peaks)     # FP32 CUDA-core updates
    assert up["peak"] == pytest.approx(bench.FP32_ALU_PEAK_GFLOPS)
    up64 = bench.class_roofline("update", st, "fp64", peaks)
    assert up64["peak"] == pytest.approx(bench.FP64_ALU_PEAK_GFLOPS)
    assert bench.class_roofline("trsm", dict(st, ms=0.0), "tf32", peaks).get("frac") is None


def test_peaks_come_from_the_measured_file_when_present():
    p = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        assert p["source"] == "of measured" and p["hbm_gbs"] == float(m["hbm_gbs"])
    else:
        assert p["source"] == "of fallback"
    assert set(bench.DTYPES) == {"fp64", "fp32", "tf32", "bf16"}


def test_solve_roofline_arithmetic_and_info_keys():
    from paper_1405_2636_gb300 import spx
    keys = spx.spx_info().as_dict()        # the binding's info dictionary
    for k in ("factor_bytes", "nnz_a", "n", "solve_ms"):
        assert k in keys
    peaks = {"hbm_gbs": 5000.0, "bf16_tflops": 2000.0, "source": "of measured"}
    info = {"factor_bytes": 7e8, "nnz_a": 1.8e6, "n": 262144, "solve_ms": 20.0}
    r = bench.solve_roofline(info, 16, 3, peaks)
    expect = 4 * 2 * 7e8 + 4 * (20 * 1.8e6 + 3 * 8 * 262144 * 16)
    assert r["sweep_pairs"] == 4 and r["algorithmic_bytes"] == pytest.approx(expect)
    assert r["achieved"] == pytest.approx(expect / 0.02 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0) and r["bound"] == "hbm"
    r0 = bench.solve_roofline(info, 16, 0, peaks)        # FP64: one sweep pair, no residual
    assert r0["algorithmic_bytes"] == pytest.approx(2 * 7e8)
    assert "frac" not in bench.solve_roofline(dict(info, solve_ms=0.0), 16, 0, peaks)
