"""bench.py's reference arm (the float64 CPU oracle) and its output contract,
on the CPU: one JSON line with the metric, a frames/s value, the oracle's
cpu_baseline record and an e2e record; under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--n-target", "2000"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference"
    assert rec["unit"] == "frames/s" and rec["value"] > 0 and rec["higher_is_better"] is True
    assert rec["config"]["workload"] == "face_shell_2k"
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"]
    assert cb["sample"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_batch_rooflines_arithmetic():
    # the roofline entries bench.py reports, from synthetic per-class event
    # times: achieved = work / average launch time, frac = achieved / peak
    sys.path.insert(0, ROOT)
    import bench
    T, n, n2, nb = 1000, 300, 40, 4
    info = {"T": T, "n": n, "n2": n2, "factor_nnz": 5000, "n_levels": 5, "n_free": 280}
    bprof = {"frames": nb, "stats": [{"iterations": 10, "sum_nc3": 8000.0}] * nb,
             "classes": {"local_step": (2, 4.0), "sigma_gemv": (2, 0.2), "reduced": (10, 5.0),
                         "detect": (0, 0.0)}}
    rl = {r["kernel_class"]: r for r in bench.batch_rooflines(bprof, info)}
    assert "detect" not in rl                       # classes without launches are left out
    loc = rl["local_step"]
    assert loc["bound"] == "alu" and loc["unit"] == "TFLOP/s"
    ach = bench.LOCAL_FLOP_PER_TET * T * nb / (2.0e-3) / 1e12
    assert abs(loc["achieved"] - ach) <= 1e-12 * ach
    assert abs(loc["frac"] - ach / bench.FP32_TFLOPS_PEAK) <= 1e-12
    assert abs(loc["traffic"] - bench.LOCAL_DRAM_BYTES_PER_TET * T * nb) <= 1e-6
    tc = rl["sigma_gemv"]
    nr = (3 * nb + 31) // 32 * 32
    assert tc["bound"] == "tensor"
    assert abs(tc["achieved"] - 3 * 2.0 * n2 * n2 * nr / 0.1e-3 / 1e12) <= 1e-9
    red = rl["reduced"]
    assert abs(red["achieved"] - 18.0 * 8000.0 * nb / 10 / 0.5e-3 / 1e12) <= 1e-12
    assert bench.dominant_roofline(list(rl.values()))["kernel_class"] == "local_step"
