"""GPU tests of the block scheduler (persistent kernel), CUDA graphs, batches
of uneven solves and the autotuner.

The scheduler is section 3.1.4's push/pop scheduler with section 3.1.2's
dependencies moved onto the device: none of these choices may change a result
bit, so every test compares against the plain launch-per-sweep path (itself
pinned to the CPU oracle in test_gpu_parity.py) or the oracle directly.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2303_02543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_02543_gb300 import jacobi as J  # noqa: E402


def solver(p, dtype="f64", block=None, **opt):
    return J.Solver(p.dims, block or p.block, dtype=dtype, faces=p.faces, source=p.source, x0=p.x0, **opt)


# ---- persistent scheduler ----------------------------------------------------

@pytest.mark.parametrize("dims,block", [((300, 190), (64, 64)), ((130, 77), (100, 30)), ((40, 33, 27), (8, 8, 8)),
                                        ((70, 20, 30), (64, 7, 9)), ((1, 1), (1, 1))])
@pytest.mark.parametrize("rows", [1, 32])
def test_persistent_f64_sweeps_bit_exact(dims, block, rows):
    p = inputs.make_problem(dims, block, 71, boundary="uniform", source="normal", x0="uniform")
    ref = oracle.sweeps(p.dims, p.faces, p.source, p.x0, 13)
    with solver(p, schedule=1, rows_f64=rows) as s:
        s.sweep(13)
        assert np.array_equal(s.field(), ref)


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("dims,block", [((60, 45), (32, 16)), ((16, 14, 12), (8, 7, 6))])
@pytest.mark.parametrize("graph", [0, 1])
def test_persistent_refine_solve_matches_oracle(dtype, e16, r16, dims, block, graph):
    p = inputs.make_problem(dims, block, 72, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 20,
                                             e_bf16=e16, r_bf16=r16)
    with solver(p, dtype=dtype, refine_period=20, schedule=1, graph=graph) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
        replays = s.profile("graph")[1]
    assert st == J.OK and st_o == oracle.OK
    assert sw == sw_o and np.array_equal(x, x_o)
    assert (replays > 0) == bool(graph)


@pytest.mark.parametrize("schedule,graph", [(0, 1), (1, 0), (1, 1)])
def test_f64_solve_schedules_match_oracle(schedule, graph):
    p = inputs.make_problem((48, 40), (16, 16), 73, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, rel_o = oracle.solve(p.dims, p.faces, p.source, None, 1e-7, 10 ** 6, 25)
    with solver(p, check_every=25, schedule=schedule, graph=graph) as s:
        st, sw, rel = s.solve(1e-7, 10 ** 6)
        x = s.field()
    assert st == J.OK and sw == sw_o and np.array_equal(x, x_o)


def test_persistent_wait_runs_out_and_reports_timeout():
    """A wait that can never be satisfied (test hook) ends with
    JACOBI_ERR_TIMEOUT after its bounded spin; the GPU stays usable."""
    p = inputs.make_problem((128, 96), (32, 32), 74, boundary="uniform", source="normal", x0="uniform")
    with solver(p, dtype="f32_refine", schedule=1, poison_wait=1, spin_limit=2000) as s:
        with pytest.raises(J.JacobiError) as e:
            s.solve(1e-8, 100)
        assert e.value.status == J.ERR_TIMEOUT
    with solver(p, schedule=1, poison_wait=1, spin_limit=2000) as s:
        s.sweep(3)
        with pytest.raises(J.JacobiError) as e:
            s.residual()  # the next synchronising call reports it
        assert e.value.status == J.ERR_TIMEOUT
    # a fresh context works
    with solver(p, schedule=1) as s:
        s.sweep(4)
        assert np.array_equal(s.field(), oracle.sweeps(p.dims, p.faces, p.source, p.x0, 4))


# ---- batches: alone vs in the mix -------------------------------------------

def uneven_problems(count, seed, scale):
    return inputs.batched_2d(seed=seed, count=count, lo=64, hi=2048, block=128, size_scale=scale)


@pytest.mark.parametrize("dtype", ["f32_refine", "f64"])
@pytest.mark.parametrize("schedule,graph", [(0, 0), (1, 1)])
def test_batch_alone_equals_mix(dtype, schedule, graph):
    probs = uneven_problems(6, 81, 0.05)   # sides about 3..100, uneven, with remainders
    tol = 1e-8 if dtype != "f64" else 1e-6
    with J.Batch(probs, dtype=dtype, refine_period=20, check_every=20, schedule=schedule, graph=graph) as b:
        st, res = b.solve(tol, 10 ** 6)
        mix = [b.field(i) for i in range(len(probs))]
    assert st == J.OK
    for i, p in enumerate(probs):
        with J.Batch([p], dtype=dtype, refine_period=20, check_every=20) as b1:
            st1, r1 = b1.solve(tol, 10 ** 6)
            alone = b1.field(0)
        assert st1 == J.OK
        assert r1[0][1] == res[i][1], (i, r1[0], res[i])      # same sweep count
        assert np.array_equal(alone, mix[i])                  # same field, bit for bit
        assert oracle.relative_residual(p.dims, p.faces, p.source, mix[i]) <= tol * (1 + 1e-9)


def test_batch_matches_oracle_per_problem():
    probs = uneven_problems(4, 82, 0.04)
    with J.Batch(probs, dtype="f32_refine", refine_period=20, schedule=1, graph=1) as b:
        st, res = b.solve(1e-8, 10 ** 6)
        for i, p in enumerate(probs):
            st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 20)
            assert res[i][1] == sw_o
            assert np.array_equal(b.field(i), x_o)


def test_batch_rejects_mixed_ndim_and_single_grid_calls():
    a = inputs.make_problem((20, 10), (10, 10), 83, source="normal")
    c = inputs.make_problem((6, 5, 4), (3, 5, 4), 84, source="normal")
    with pytest.raises(J.JacobiError):
        J.Batch([a, c])
    with J.Batch([a, a]) as b:
        with pytest.raises(J.JacobiError):
            J.jacobi_residual(b.h)


# ---- autotuner ------------------------------------------------------------------

def test_autotune_keeps_results_and_writes_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("JACOBI_TUNE_CACHE", str(cache))
    p = inputs.make_problem((200, 150), (64, 64), 85, boundary="uniform", source="normal", x0="zero")
    with solver(p, dtype="f32_refine", refine_period=20) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        ref = s.field()
    with solver(p, dtype="f32_refine", refine_period=20, autotune=1) as s:
        st2, sw2, rel2 = s.solve(1e-8, 10 ** 6)
        assert sw2 == sw and np.array_equal(s.field(), ref)
    assert cache.exists() and "rows" in cache.read_text()
    with solver(p, dtype="f32_refine", refine_period=20, autotune=1) as s:  # served from the cache
        st3, sw3, _ = s.solve(1e-8, 10 ** 6)
        assert sw3 == sw and np.array_equal(s.field(), ref)
    with solver(p, autotune=1, check_every=10) as s:  # FP64 tuning must leave the iterate untouched
        s.sweep(0)
        st4, sw4, _ = s.solve(1e-3, 10 ** 5)
        st5, x5, sw5, _ = oracle.solve(p.dims, p.faces, p.source, None, 1e-3, 10 ** 5, 10)
        assert sw4 == sw5 and np.array_equal(s.field(), x5)


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("graph", [0, 1])
def test_split_outer_step_3d_bit_exact(dtype, e16, r16, graph):
    """The 3D outer step as x + e over the layout then the residual pass gives
    the bits of the fused pass and of the oracle, alone and in a batch of
    uneven 3D solves (several slots of the apply kernel's grid)."""
    probs = [inputs.make_problem(d, b, 90 + i, boundary="uniform", source="normal", x0="zero")
             for i, (d, b) in enumerate([((20, 17, 13), (8, 9, 5)), ((9, 30, 11), (9, 16, 4)), ((33, 5, 7), (32, 5, 7))])]
    fields = {}
    for split in (0, 1):
        with J.Batch(probs, dtype=dtype, refine_period=10, outer_split=split, graph=graph) as b:
            st, res = b.solve(1e-8, 10 ** 6)
            assert st == J.OK
            fields[split] = ([b.field(i) for i in range(len(probs))], [r[1] for r in res])
    assert fields[0][1] == fields[1][1]
    for i, p in enumerate(probs):
        assert np.array_equal(fields[0][0][i], fields[1][0][i])
        st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 10,
                                                 e_bf16=e16, r_bf16=r16)
        assert fields[1][1][i] == sw_o
        assert np.array_equal(fields[1][0][i], x_o)


@pytest.mark.parametrize("dtype", ["f32_refine", "f64"])
def test_batch_retune_after_compaction_keeps_results(dtype, tmp_path, monkeypatch):
    """With the autotuner on, a batch whose solves retire at different times is
    re-tuned for the remaining ones once they are a minority of the points;
    every result is still the one the solve gives alone."""
    monkeypatch.setenv("JACOBI_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    probs = uneven_problems(6, 83, 0.06)
    tol = 1e-8 if dtype != "f64" else 1e-6
    with J.Batch(probs, dtype=dtype, refine_period=20, check_every=20, autotune=1, graph=1) as b:
        st, res = b.solve(tol, 10 ** 6)
        mix = [b.field(i) for i in range(len(probs))]
    assert st == J.OK
    for i, p in enumerate(probs):
        with J.Batch([p], dtype=dtype, refine_period=20, check_every=20) as b1:
            st1, r1 = b1.solve(tol, 10 ** 6)
            alone = b1.field(0)
        assert st1 == J.OK and r1[0][1] == res[i][1]
        assert np.array_equal(alone, mix[i])
    lines = (tmp_path / "tune.jsonl").read_text().splitlines()
    assert len(lines) >= 2  # the first tuning and at least one re-tuning
