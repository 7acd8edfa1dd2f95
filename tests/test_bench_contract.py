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


def test_serving_leg_counts_censored_requests_in_the_all_request_bound(monkeypatch):
    """The serving leg's host logic against a fake server: completed requests
    give p50/p99 over their latencies; requests still running at the deadline
    are censored and enter the all-request percentiles with their waiting
    time so far (a lower bound)."""
    import types
    sys.path.insert(0, ROOT)
    import bench
    from paper_2303_02543_gb300 import inputs
    from paper_2303_02543_gb300 import jacobi as J

    arrivals = [types.SimpleNamespace(t=0.0, problem=types.SimpleNamespace(points=100)) for _ in range(4)]
    monkeypatch.setattr(inputs, "serving_stream", lambda **kw: arrivals)

    class FakeServer:
        def __init__(self, *a, **kw):
            self.n = 0

        def submit(self, problem, tol, max_sweeps):
            self.n += 1
            return self.n

        def stats(self):
            return {"completed": 2, "rejected": 0, "steps": 7, "evictions": 0, "resumed": 0}

        def poll(self, ticket, want_field=True):
            # tickets 1 and 2 finished in 0.1 s and 0.3 s; 3 and 4 still run
            return (J.OK, 10, 1e-9, 0.1 * (2 * ticket - 1), None) if ticket <= 2 else None

        def close(self):
            pass

    monkeypatch.setattr(J, "Server", FakeServer)
    import torch
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    leg = bench.serving_leg(1.0, 0.0, 256, 64, 0, grace=0.05)
    assert leg["requests"] == 4 and leg["completed"] == 2 and leg["censored"] == 2
    assert abs(leg["p50_ms"] - 300.0) < 1e-6 and abs(leg["p99_ms"] - 300.0) < 1e-6
    # the censored requests have waited at least the grace period
    assert leg["p99_ms_all_lower_bound"] >= 50.0 and leg["p50_ms_all_lower_bound"] >= 100.0
    assert leg["glups"] > 0 and leg["steps"] == 7
