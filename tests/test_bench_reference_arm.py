"""The oracle arm of bench.py (`--impl reference`): runs on host cores only,
prints one JSON line with the benchmark's metric, config and the
cpu_baseline / e2e objects, and needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_ref(*extra):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "3", *extra],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = run_ref()
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert "workload" in d["config"] and "mixed" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == os.cpu_count() and cb["value"] == d["value"] and cb["sample"]
    assert cb["host"]["cpu_count"] == os.cpu_count() and cb["host"]["cpu_model"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_workload():
    d = run_ref("--workload", "hubbard2")
    assert d["config"]["workload"].startswith("2-orbital")
    assert d["impl"] == "reference" and d["value"] > 0
    assert "2-orbital" in d["config"]["workload"] or "hubbard" in d["config"]["workload"].lower()


def test_oracle_worker_thread_count_and_results():
    """The cpu_baseline leg's child processes run with the BLAS / OpenMP
    thread count fixed in their environment, and return the oracle's value
    of every chain of the first pass (used for the error report)."""
    sys.path.insert(0, ROOT)
    import bench
    spec = {"workload": "hubbard2", "first": 8, "min_s": 0.0, "n_min": 8}
    r = bench.oracle_subprocess(spec, threads=1)
    assert r["count"] == 8 and len(r["results"]) == 8 and r["rate"] > 0
    st, la, re, im = r["results"]["0"]
    assert st == "ok" and abs(abs(complex(re, im)) - 1.0) < 1e-12
    assert all(v == "1" for v in r["blas_threads"].values())
