"""The benchmark's contract, checked on the CPU: the reference arm's JSON line (the oracle on a
bounded sample of the 128-orbital workload), the silent non-zero ranks under torchrun, and the
pure helpers behind the roofline fields."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                       text=True, cwd=ROOT, env=e, timeout=900)
    return r


def test_reference_arm_prints_one_complete_json_line():
    r = run_bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-sample", "64")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "c3-mgo64-96"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_silently():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--ref-sample", "16",
                  env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_algorithmic_bytes_per_evaluation():
    """64 gathered coefficients per table, five outputs and the 24-byte position shared by the
    orbitals: 532.2 B (FP32, two tables), 276.2 B (BF16), 1064.2 B (FP64), 128 orbitals."""
    assert bench.algorithmic_bytes_per_eval("f32", 2, 128) == pytest.approx(2 * 64 * 4 + 20 + 24 / 128)
    assert bench.algorithmic_bytes_per_eval("bf16", 2, 128) == pytest.approx(2 * 64 * 2 + 20 + 24 / 128)
    assert bench.algorithmic_bytes_per_eval("f64", 2, 128) == pytest.approx(2 * 64 * 8 + 40 + 24 / 128)
    assert bench.algorithmic_bytes_per_eval("df64", 1, 128) == pytest.approx(64 * 8 + 40 + 24 / 128)


def test_l1_roofline_uses_the_measured_probe_rate():
    l1 = {"gbs": 36000.0, "bytes_per_clk_per_sm": 120.0, "sm_mhz": 1974.0}
    r = bench.l1_roofline(40.0e9, 1.0e-3, l1)
    assert r["bound"] == "l1" and r["peak"] == 36000.0
    assert r["achieved"] == pytest.approx(40.0e9 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 36000.0)


def test_cache_rooflines_pick_the_binding_level():
    l1 = {"gbs": 80000.0}
    l2 = {"gbs": 20000.0}
    top, lv = bench.cache_rooflines(40.0e9, 15.0e9, 3.0e9, 1.0e-3, l1, l2, 6800.0, "measured")
    assert lv["l1"]["frac"] == pytest.approx(0.5)
    assert lv["l2"]["frac"] == pytest.approx(0.75)
    assert lv["hbm"]["frac"] == pytest.approx(3000.0 / 6800.0)
    assert top["bound"] == "l2" and top["frac"] == lv["l2"]["frac"]
    top, lv = bench.cache_rooflines(40.0e9, None, None, 1.0e-3, l1, l2, 6800.0, "measured")
    assert set(lv) == {"l1"} and top["bound"] == "l1"


def test_precision_report_on_hand_made_outputs():
    """Errors per output against the unrounded and the rounded reference, and the kinetic-energy
    change: a Laplacian error of 0.01 at every sample of an orbital with phi = 1 moves its T_n by
    -1/2 * 0.01 = -5 mHa."""
    P, O = 8, 3
    val = np.ones((P, O))
    grad = np.zeros((P, 3, O))
    grad[:, 0, :] = 2.0
    lap = np.full((P, O), -4.0)
    ref = (val, grad, lap)
    got = (val.copy(), grad.copy(), lap.copy())
    got[2][:, 1] += 0.01
    got[1][3, 0, 2] += 0.002
    r = bench.precision_report("f32", got, ref, ref, "hand-made")
    assert r["max_rel_err_vs_fp64"]["val"] == 0.0
    assert r["max_rel_err_vs_fp64"]["grad"] == pytest.approx(0.001)
    assert r["max_rel_err_vs_fp64"]["lap"] == pytest.approx(0.0025)
    assert r["dT_mHa"] == pytest.approx(5.0)
    assert r["T_max_Ha"] == pytest.approx(2.0)
    assert r["ok"] is False and r["tolerance"] == 2e-6


def test_both_arms_report_the_same_workload_config():
    from paper_1309_6250_gb300 import inputs
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--ref-sample", "16")
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["config"] == bench.workload_config(inputs.make_workload("c3"))


def test_traffic_is_dropped_when_the_kernel_source_changes(monkeypatch):
    """DRAM bytes from the committed ncu capture are reported only while the kernel source hash
    matches the one the capture was taken on."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        entries = json.load(f)
    key, entry = next(iter(entries.items()))
    if entry["kernel_source_sha"] == bench.kernel_source_hash():
        assert bench.load_traffic(key)["dram"] == entry["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda sources=None: "0000000000000000")
    assert bench.load_traffic(key) is None
    assert bench.load_traffic("no/such/key") is None
