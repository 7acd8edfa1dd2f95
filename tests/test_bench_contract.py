"""bench.py's JSON line contract, checked on the CPU through its reference
arm (the oracle on the host cores): one line with the keys every arm prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line_with_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "laplace2d_256"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "GLUP/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "laplace2d_256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_cpu_baseline_leg_reports_all_cores_and_one_thread():
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    p, _, _ = bench.make_workload("laplace2d_256")
    try:
        cb = bench.cpu_baseline(p, "laplace2d_256")
    finally:
        # the oracle keeps the thread count it was last given: hand back all of them
        oracle.sweeps((2, 2), None, None, None, 1, threads=threads)
    assert oracle.max_threads() == threads
    assert cb["kind"] == "oracle" and cb["unit"] == "GLUP/s" and cb["value"] > 0 and cb["cores"] >= 1
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0
