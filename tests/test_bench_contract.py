"""The benchmark's reference arm keeps the JSON-line contract (CPU only): one line, the headline
keys, the reference marker, a CPU-baseline description, and an end-to-end entry without
host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"]:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "seq_320x240_n256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_clock_summary_reads_median_and_throttle_reasons():
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.lines = ["0, 1200, 2070, 500, 0x8, Active, Not Active, Not Active, Not Active"]
    assert bench.ClockSampler.summary(cs)["reasons"] == ["hw_slowdown"]


def test_traffic_reported_only_for_the_captured_kernel_source_and_workload():
    sys.path.insert(0, ROOT)
    import bench
    c = dict(bench.CHOL_TRAFFIC)
    try:
        bench.CHOL_TRAFFIC = dict(c, chol_sha256=bench._chol_source_digest())
        assert bench._chol_traffic(c["precision"], c["streams"]) == c["bytes"]
        assert bench._chol_traffic(0, c["streams"]) is None
        assert bench._chol_traffic(c["precision"], 8) is None
        bench.CHOL_TRAFFIC = dict(c, chol_sha256="0" * 16)     # another kernel source
        assert bench._chol_traffic(c["precision"], c["streams"]) is None
    finally:
        bench.CHOL_TRAFFIC = c
