"""Host logic of bench.py, on the CPU: the reference arm's JSON line (the
FP64 oracle timed on host cores), the clock-sample summary that decides
whether a run is kept, and the roofline arithmetic built on the committed
ncu record."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--n-samp", "8192",
                        "--ref-budget-s", "0.5"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["n_samp"] == 8192


def test_reference_arm_other_ranks_print_nothing(capsys):
    import argparse
    ns = argparse.Namespace(n_samp=8192, n_dm=4096, steps=1, warmup=0, ref_budget_s=0.5)
    assert bench.run_reference(ns, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


def test_clock_summary():
    q = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    lines = [q.format(sm=2070, hw="Not Active", pc="Not Active"),
             q.format(sm=2055, hw="Not Active", pc="Active"),
             q.format(sm=2070, hw="Not Active", pc="Not Active"),
             "garbage line", "0, [N/A], 2070, 1, 0x0, a, b, c, d"]
    s = bench.Clocks.parse("\n".join(lines))
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    s = bench.Clocks.parse(q.format(sm=1200, hw="Active", pc="Not Active"))
    assert s["reasons"] == ["hw_slowdown"] and s["sm_mhz"] == 1200.0
    assert bench.Clocks.parse("") is None


def test_roofline_arithmetic_from_the_ncu_record():
    kv = bench._recorded()
    if kv is None:
        pytest.skip("the committed ncu record is for another kernel source")
    n, c = int(kv["samples"]), int(kv["candidates"])
    rd, wr = float(kv["dram_read_bytes"]), float(kv["dram_write_bytes"])
    assert bench.recorded_traffic(n, c) == int(rd + wr)
    # reads scale with samples, writes with candidates
    assert bench.recorded_traffic(8 * n, 2 * c) == int(8 * rd + 2 * wr)
    inst = float(kv["warp_instructions"])
    assert bench.recorded_instructions(8 * n) == pytest.approx(8 * inst)
    r = bench.issue_roofline(n, 2.0)
    assert r["bound"] == "issue" and r["unit"] == "Twarp-inst/s"
    assert r["achieved"] == pytest.approx(inst / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = json.load(f).get("sm_max_mhz") or mhz
    except OSError:
        pass
    assert r["peak"] == pytest.approx(152 * 4 * mhz * 1e6 / 1e12)
