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
    assert d["config"]["workload"] == "batched_mixed_64"
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
    c = bench.FACTOR_TRAFFIC
    try:
        bench.FACTOR_TRAFFIC = {"chol_sha256": bench._chol_source_digest(),
                                "workload": bench.WORKLOAD, "bytes": {"tc128p": 123}}
        assert bench._factor_traffic(bench.WORKLOAD, "tc128p") == 123
        assert bench._factor_traffic("seq_320x240_n256", "tc128p") is None
        assert bench._factor_traffic(bench.WORKLOAD, "tc128") is None      # another kernel
        bench.FACTOR_TRAFFIC = dict(bench.FACTOR_TRAFFIC, chol_sha256="0" * 16)   # other source
        assert bench._factor_traffic(bench.WORKLOAD, "tc128p") is None
        bench.FACTOR_TRAFFIC = None
        assert bench._factor_traffic(bench.WORKLOAD, "tc128p") is None
    finally:
        bench.FACTOR_TRAFFIC = c


def test_error_sample_and_comparison():
    """The oracle sample takes the fewest-node problem of each template size; the comparison
    reports positions, the last cost and mask bits outside the listed band."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from synth.workloads import mixed_problems
    ps = mixed_problems(64)
    ks = bench.error_sample(ps)
    assert len(ks) == 3 and len({ps[k].cfg.W for k in ks}) == 3
    for k in ks:
        assert ps[k].cfg.N == min(p.cfg.N for p in ps if p.cfg.W == ps[k].cfg.W)
    g = np.zeros((2, 3))
    ref = {"g": g, "pos": np.array([[1.0, 0, 0], [0, 0, 0]]), "cost": np.array([5.0, 4.0]),
           "mask": np.array([True, False, True]), "kept": np.array([True]),
           "d": np.array([[0.5, 2.0 + 1e-9, 0.1]]), "score": np.array([3.0])}
    gpu = {"t": np.array([[1.0, 0, 0], [0, 0, 3e-4]]), "cost": 4.0004,
           "mask": np.array([True, True, False])}
    c = bench.compare(gpu, ref, 2.0)
    assert abs(c["max_err_mm"] - 3e-4) < 1e-15 and abs(c["cost_rel_err"] - 1e-4) < 1e-12
    assert c["mask_bits_differing"] == 1     # match 1 sits in the band around H, match 2 counts


def test_phase_rooflines_count_the_algorithmic_bytes():
    """The bench line's phase HBM fractions: per iteration the linearisation moves 6 sum n^2 B of
    matrix writes plus 64 B per template point, the solves 4 sum n^2 B per solve (1 + refinement
    steps) and per refinement residual."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench._phase_rooflines([40.0, 130.0, 50.0, 0.3], sum_n2=1e9, points=8e6, iters=10,
                               refine_steps=2, hbm_gbs=6000.0)
    lin = 10 * (6e9 + 64 * 8e6)
    sol = 10 * 4e9 * 5
    assert r["linearize"]["bytes_per_step"] == int(lin)
    assert r["solve_refine"]["bytes_per_step"] == int(sol)
    assert abs(r["linearize"]["achieved_gbs"] - lin / 0.040 / 1e9) < 0.1
    assert abs(r["solve_refine"]["frac"] - sol / 0.050 / 1e9 / 6000.0) < 1e-4
    json.dumps(r)
