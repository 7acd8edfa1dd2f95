"""The N > 1 path on the CPU (gloo, world size 2): bench.py's rank helpers and
its reference arm under torch.distributed.run.  Every rank solves its own copy
of the problem (weak scaling, no collective on the data path); the barrier and
the max over ranks only bracket the timed region."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, _ = bench.dist_setup(None)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    m = bench.max_over_ranks(float(10 + rank), w)
    out.put((rank, m))
    torch.distributed.destroy_process_group()


def test_rank_helpers_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 11.0), (1, 11.0)]


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "laplace2d_256"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2


def _failing_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), JACOBI_PG_TIMEOUT_S="20")
    sys.path.insert(0, ROOT)
    import time

    import bench
    bench.dist_setup(None)
    if rank == 1:
        os._exit(3)  # this rank fails between steps: it never reaches the barrier
    t0 = time.time()
    try:
        bench.barrier(world)
        out.put(("no error", time.time() - t0))
    except Exception as e:  # noqa: BLE001 - the error itself is the result
        out.put((type(e).__name__, time.time() - t0))
    out.close()
    out.join_thread()  # flush the result before leaving without teardown
    os._exit(0)


def test_a_failed_rank_ends_the_others_barrier_with_an_error():
    """Failure detection on the host: when one rank dies between steps, the
    surviving rank's next collective raises (peer gone, or the short
    process-group timeout) instead of waiting for ever."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    kind, seconds = q.get(timeout=10)
    assert kind != "no error" and seconds < 60
