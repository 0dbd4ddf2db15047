"""The benchmark's reference arm (the oracle timed on the host cores) runs
without a GPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "deform3d", "--n", "10", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "sample" in cb
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("deform3d")


def test_cpu_baseline_leg_with_one_thread():
    """The benchmark's cpu_baseline leg: the oracle on all host cores, the CPU
    model, and one step on a single thread beside it."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1305_3417_gb300 import inputs as I
    w = I.make_workload("deform3d", n=8)
    base, _ = bench.cpu_baseline(w, steps=1, one_thread=True)
    assert base["kind"] == "oracle" and base["value"] > 0 and base["cores"] >= 1
    assert isinstance(base["cpu_model"], str) and base["cpu_model"]
    one = base["one_thread"]
    assert one["cores"] == 1 and one["value"] > 0
