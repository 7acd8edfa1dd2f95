"""Serving: continuous batching under an HBM budget.

Requests that arrive while others run are admitted as slots and memory free
up; every result must equal the same solve run alone (same refine_period),
bit for bit, and the budget must bound the resident state.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2303_02543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_02543_gb300 import jacobi as J  # noqa: E402

K = 20
MAXS = 20 * 50000


def alone(p, dtype="f32_refine"):
    with J.Solver(p.dims, p.block, dtype=dtype, faces=p.faces, source=p.source, x0=p.x0, refine_period=K,
                  schedule=1) as s:
        st, sw, rel = s.solve(1e-8, MAXS)
        return st, sw, s.field()


def mixed_requests():
    return [inputs.make_problem((90, 70), (32, 32), 91, boundary="uniform", source="normal"),
            inputs.make_problem((14, 12, 10), (8, 8, 8), 92, boundary="uniform", source="normal"),
            inputs.make_problem((160, 40), (64, 40), 93, boundary="uniform", source="normal"),
            inputs.make_problem((9, 9, 9), (9, 9, 9), 94, boundary="uniform", source="normal"),
            inputs.make_problem((33, 120), (33, 64), 95, boundary="uniform", source="normal"),
            inputs.make_problem((20, 7, 16), (10, 7, 8), 96, boundary="uniform", source="normal")]


@pytest.mark.parametrize("dtype", ["f32_refine", "bf16_refine"])
def test_results_equal_alone_with_staggered_arrivals(dtype):
    probs = mixed_requests()
    with J.Server(dtype, budget_bytes=256 << 20, max_slots=8, refine_period=K) as srv:
        tickets = [srv.submit(p, 1e-8, MAXS) for p in probs[:3]]
        time.sleep(0.02)                      # the first ones are running when the rest arrive
        tickets += [srv.submit(p, 1e-8, MAXS) for p in probs[3:]]
        outs = []
        for t in tickets:
            assert srv.wait(t, 120.0)
            outs.append(srv.poll(t))
        stats = srv.stats()
    assert stats["completed"] == len(probs) and stats["admitted"] == len(probs)
    for p, (st, sw, rel, secs, field) in zip(probs, outs):
        st1, sw1, x1 = alone(p, dtype)
        assert st == J.OK and st1 == J.OK
        assert sw == sw1
        assert np.array_equal(field, x1)
        assert oracle.relative_residual(p.dims, p.faces, p.source, field) <= 1e-8 * (1 + 1e-9)


def test_budget_bounds_resident_state_and_queues():
    # about 2.8 MB of state each (x twice, f, e twice, r, faces, partials,
    # tables): an 8.5 MB arena holds two at a time, never three
    probs = [inputs.make_problem((256, 256), (64, 64), 100 + i, boundary="uniform", source="normal") for i in range(5)]
    with J.Server("f32_refine", budget_bytes=int(8.5 * (1 << 20)), max_slots=8, refine_period=K) as srv:
        tickets = [srv.submit(p, 1e-8, MAXS) for p in probs]
        peak = 0
        while True:
            s = srv.stats()
            peak = max(peak, s["active"])
            assert s["bytes_in_use"] <= s["budget_bytes"]
            if s["completed"] == len(probs):
                break
            time.sleep(0.001)
        results = [srv.poll(t) for t in tickets]
    assert 1 <= peak < len(probs)
    for p, r in zip(probs, results):
        assert r[0] == J.OK
        assert np.array_equal(r[4], alone(p)[2])


def test_request_larger_than_budget_is_refused():
    with J.Server("f32_refine", budget_bytes=4 << 20, max_slots=4) as srv:
        with pytest.raises(J.JacobiError) as e:
            srv.submit(inputs.make_problem((1024, 1024), (128, 128), 110, source="normal"), 1e-8, MAXS)
        assert e.value.status == J.ERR_BUSY
        assert srv.stats()["rejected"] == 1


def test_short_request_overtakes_long_one():
    """Continuous batching: a small solve submitted after a big one is
    admitted while the big one runs and finishes first."""
    big = inputs.make_problem((400, 400), (128, 128), 120, boundary="uniform", source="normal")
    small = inputs.make_problem((24, 24), (24, 24), 121, boundary="uniform", source="normal")
    with J.Server("f32_refine", budget_bytes=512 << 20, max_slots=4, refine_period=K) as srv:
        tb = srv.submit(big, 1e-8, MAXS)
        time.sleep(0.01)
        ts = srv.submit(small, 1e-8, MAXS)
        assert srv.wait(ts, 60.0)
        assert srv.poll(tb, want_field=False) is None  # the big one is still running
        rs = srv.poll(ts)
        assert srv.wait(tb, 300.0)
        rb = srv.poll(tb)
    assert rs[0] == J.OK and rb[0] == J.OK and rs[3] < rb[3]
    assert np.array_equal(rs[4], alone(small)[2]) and np.array_equal(rb[4], alone(big)[2])


def _smallest_accepted_budget(problem, lo=1 << 20, hi=64 << 20):
    """Smallest budget (to 1 KiB) whose server accepts the request at submit."""
    def accepted(budget):
        with J.Server("f32_refine", budget_bytes=budget, max_slots=8, refine_period=K) as srv:
            try:
                srv.submit(problem, 1e300, 0)      # done at its first check
            except J.JacobiError as e:
                assert e.status == J.ERR_BUSY
                return False
            return True
    assert accepted(hi) and not accepted(lo)
    while hi - lo > 1024:
        mid = (lo + hi) // 2
        lo, hi = (lo, mid) if accepted(mid) else (mid, hi)
    return hi


def test_tight_arena_retires_and_admits_without_device_temporaries():
    """Arenas around the size that holds three solves with almost nothing
    left over: admission and retirement take no device memory from the arena,
    so every solve completes, equal to the same solve run alone, however
    little room the resident ones leave."""
    p = inputs.make_problem((128, 128), (32, 32), 130, boundary="uniform", source="normal")
    ref = alone(p)[2]
    # the submit check accepts a request whose estimate b satisfies
    # b + b/16 + 1 MiB <= budget
    b = (_smallest_accepted_budget(p) - (1 << 20)) * 16 // 17
    for delta in range(-32 << 10, 161 << 10, 16 << 10):
        budget = 3 * b + b // 16 + delta
        with J.Server("f32_refine", budget_bytes=budget, max_slots=8, refine_period=K) as srv:
            tickets = [srv.submit(p, 1e-8, MAXS) for _ in range(4)]
            for t in tickets:
                assert srv.wait(t, 120.0), (delta, srv.stats())
            results = [srv.poll(t) for t in tickets]
            stats = srv.stats()
        assert stats["completed"] == 4 and stats["rejected"] == 0, (delta, stats)
        for r in results:
            assert r[0] == J.OK
            assert np.array_equal(r[4], ref)


@pytest.mark.parametrize("max_slots", [1, 4096])
def test_request_near_the_budget_completes_or_is_rejected_never_stalls(max_slots):
    """A request accepted at submit is placed in an empty arena or, if its
    state and the workset's tables do not fit there, completes with
    JACOBI_ERR_OOM; the server neither stalls nor stops."""
    p = inputs.make_problem((96, 80), (32, 32), 131, boundary="uniform", source="normal")
    ref = alone(p)[2]
    one = _smallest_accepted_budget(p)
    for budget in (one, one + (64 << 10), one + (256 << 10)):
        with J.Server("f32_refine", budget_bytes=budget, max_slots=max_slots, refine_period=K) as srv:
            t = srv.submit(p, 1e-8, MAXS)
            assert srv.wait(t, 60.0), srv.stats()
            st, sw, rel, secs, field = srv.poll(t)
            stats = srv.stats()
            if st == J.OK:
                assert np.array_equal(field, ref) and stats["rejected"] == 0
            else:
                assert st == J.ERR_OOM and sw == 0 and stats["rejected"] == 1
            # the server still serves: a small request after it completes
            q = inputs.make_problem((8, 8), (8, 8), 132, boundary="uniform", source="normal")
            t2 = srv.submit(q, 1e-8, MAXS)
            assert srv.wait(t2, 60.0), srv.stats()
            assert srv.poll(t2)[0] == J.OK


def test_options_are_fixed_by_the_first_submit():
    with J.Server("f32_refine", budget_bytes=64 << 20, max_slots=4) as srv:
        t = srv.submit(inputs.make_problem((16, 16), (16, 16), 133, source="normal"), 1e-8, MAXS)
        assert J.load().jacobi_server_set_option(srv.h, b"refine_period", 10) == J.ERR_BUSY
        assert srv.wait(t, 60.0)
        srv.poll(t)
        # still fixed after the queue drained and the solve retired
        assert J.load().jacobi_server_set_option(srv.h, b"refine_period", 10) == J.ERR_BUSY


@pytest.mark.parametrize("dtype", ["f32_refine", "bf16_refine"])
def test_evicted_solve_resumes_bit_identical(dtype):
    """Serving under HBM pressure: with one slot, small requests that queue
    behind a long solve make the server evict it to host memory; they run and
    finish first, and the long solve, admitted again, returns the same field
    and sweep count as a solve that was never evicted, bit for bit."""
    long_ = inputs.make_problem((200, 160), (64, 64), 130, boundary="uniform", source="normal")
    shorts = [inputs.make_problem((40, 30), (20, 30), 131 + i, boundary="uniform", source="normal") for i in range(3)]
    with J.Server(dtype, budget_bytes=256 << 20, max_slots=1, refine_period=K, evict=1, evict_min_steps=5,
                  evict_wait_steps=1) as srv:
        tl = srv.submit(long_, 1e-8, MAXS)
        while srv.stats()["steps"] < 10:
            time.sleep(0.001)
        ts = [srv.submit(p, 1e-8, MAXS) for p in shorts]
        for t in ts:
            assert srv.wait(t, 120.0)
        rs = [srv.poll(t) for t in ts]
        assert srv.wait(tl, 300.0)
        rl = srv.poll(tl)
        stats = srv.stats()
    assert stats["evictions"] == 1 and stats["resumed"] == 1
    assert rl[3] > max(r[3] for r in rs)  # the long solve finished last
    for p, r in zip(shorts + [long_], rs + [rl]):
        st1, sw1, x1 = alone(p, dtype)
        assert r[0] == J.OK and st1 == J.OK
        assert r[1] == sw1
        assert np.array_equal(r[4], x1)


def test_without_eviction_small_requests_wait_for_the_slot():
    long_ = inputs.make_problem((200, 160), (64, 64), 130, boundary="uniform", source="normal")
    short = inputs.make_problem((40, 30), (20, 30), 131, boundary="uniform", source="normal")
    with J.Server("f32_refine", budget_bytes=256 << 20, max_slots=1, refine_period=K) as srv:
        tl = srv.submit(long_, 1e-8, MAXS)
        while srv.stats()["steps"] < 10:
            time.sleep(0.001)
        t = srv.submit(short, 1e-8, MAXS)
        assert srv.wait(t, 300.0) and srv.wait(tl, 300.0)
        rs, rl = srv.poll(t), srv.poll(tl)
        assert srv.stats()["evictions"] == 0
    assert rs[3] > rl[3]  # queued behind the long solve
    assert np.array_equal(rl[4], alone(long_)[2])


def test_eviction_options_are_checked():
    with J.Server("f32_refine", budget_bytes=16 << 20, max_slots=2) as srv:
        for k, v in (("evict", 2), ("evict_min_steps", 0), ("evict_wait_steps", -1), ("max_evictions", 0)):
            with pytest.raises(J.JacobiError) as e:
                J._check(J.load().jacobi_server_set_option(srv.h, k.encode(), v), None)
            assert e.value.status == J.ERR_INVALID
