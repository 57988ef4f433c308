"""bench.py's output contract, exercised on the CPU through the reference arm.

The reference arm times the oracle on the host cores and prints the same JSON
line as the GPU arm; this checks the keys and types the contract fixes, on the
small 4x4 workload (a second or two of CPU time), and that on the gradient
workload it times the gradient and reports the GPU arm's metric and unit."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_line_keys():
    d = _run("--impl", "reference", "--workload", "n16_beta8", "--steps", "2", "--warmup", "1")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "n16_beta8"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_metric_matches_workload():
    sys.path.insert(0, ROOT)
    import bench
    d = _run("--impl", "reference", "--workload", "grad_n144", "--steps", "1", "--warmup", "0")
    assert (d["metric"], d["unit"]) == bench.METRICS["grad_n144"] == ("logdet_gradients_per_second",
                                                                      "grads/s")
    assert d["impl"] == "reference" and d["value"] > 0
    # one sample is a fraction of a gradient: 2 of the M = 200 slices; a step
    # is one sample (mode B) or one sample per process of the pool (mode A)
    per = d["config"]["instances_per_step"] / (2 / 200)
    assert abs(per - round(per)) < 1e-9 and round(per) >= 1
    assert d["config"]["cpu_mode"] in ("pool", "threads")
    if d["config"]["cpu_mode"] == "threads":
        assert round(per) == 1
    assert d["cpu_baseline"]["unit"] == "grads/s"
    assert d["cpu_baseline"]["cpu_model"]
