"""Host-side parts of bench.py, on the CPU: the derived roofline peaks, the
committed ncu record of the headline KSG launch, and the reference arm's JSON
line (the FP64 oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_derived_peaks():
    pk = dict(sms=152, sm_max_mhz=2070.0, bf16_tflops_sustained=1700.0, hbm_gbs=6800.0,
              source="test")
    # 152 SMs x 128 FFMA lanes x 2 flop x 2.07 GHz, and x 64 ALU-pipe lanes
    assert bench.peak_of("fp32_flop", pk)[0] == pytest.approx(80.5478, rel=1e-5)
    assert bench.peak_of("ksg_instr", pk)[0] == pytest.approx(20.13696, rel=1e-6)
    assert bench.peak_of("fp8", pk)[0] == 2 * bench.peak_of("bf16", pk)[0] == 3400.0
    assert bench.peak_of("hbm", pk)[0] == 6800.0
    with pytest.raises(ValueError):
        bench.peak_of("fp64", pk)
    # the definition's ALU work per pair: one max and two comparisons per ordered (i, j)
    assert bench.ksg_definition_instr(100) == 3 * 100 * 99
    assert bench.ksg_definition_instr(2) == 6


def test_peaks_take_the_device_sm_count():
    assert bench.peaks(148)["sms"] == 148
    assert bench.peaks(None)["sms"] == 152


def test_headline_kernel_counters_belong_to_the_sources():
    """The ncu record of the KSG launch was captured on the current KSG
    sources (their hash is recorded), so the bench line's roofline traffic is
    a number; a change to those sources without a new capture turns it null."""
    rec = bench.kernel_counters("k_ksg_stream", bench.FOC["name"])
    assert rec is not None
    assert rec["dram_bytes"] > 0 and rec["inst_executed_per_pair"] > 0
    assert os.path.exists(os.path.join(ROOT, "profiles", rec["capture"]))
    assert bench.kernel_counters("k_no_such_kernel", bench.FOC["name"]) is None


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the FP64 oracle on a bounded sample of
    the headline workload and prints one JSON line with the contract's keys."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "point-pairs/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["metric"] == bench.METRIC and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0
    assert e2e["d2h_bytes_per_step"] == 0
