"""GPU parity at the benchmark's full sizes, in its launch configuration.

The oracle cannot rerun an 8192^2 or 512^3 solve in a test, so every run here
is checked point by point on sampled outputs, each recomputed by the oracle
on the window that holds its dependency cone (cones.py): corners, both sides
of block seams, domain edges and seeded interior points, compared bit for
bit.  The 8192^2 FP64 run is also checked on a property of the whole field:
its relative residual, recomputed by the oracle from the GPU's field.
"""
import numpy as np
import pytest

import oracle
from paper_2303_02543_gb300 import inputs
from cones import sample_points, value_at, window

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_02543_gb300 import jacobi as J  # noqa: E402

CHECK_EVERY = 50


def check_samples(p, field, radius, run, count, seed):
    for c in sample_points(p.dims, p.block, count, seed):
        wd, wf, ws, wx, idx = window(p, c, radius)
        ref = run(wd, wf, ws, wx)
        assert value_at(field, c) == value_at(ref, idx), c


@pytest.fixture(scope="module")
def poisson2d_8192():
    return inputs.poisson_2d_large()


def test_fullsize_2d_8192_f64(poisson2d_8192):
    """8192^2, 16x16 blocks of 512^2, FP64: 100 sweeps with the residual
    tested every 50, as bench.py runs it."""
    p = poisson2d_8192
    k = 100
    with J.Solver(p.dims, p.block, dtype="f64", faces=p.faces, source=p.source, x0=p.x0,
                  check_every=CHECK_EVERY, refine_period=CHECK_EVERY, profile=1) as s:
        st, sw, rel = s.solve(1e-300, k)
        field = s.field()
    assert st == J.ERR_NOT_CONVERGED and sw == k
    check_samples(p, field, k, lambda d, f, src, x0: oracle.sweeps(d, f, src, x0, k), 24, 71)
    rel_o = oracle.relative_residual(p.dims, p.faces, p.source, field)
    assert abs(rel - rel_o) <= 1e-12 * rel_o


def test_fullsize_2d_8192_f32_refine(poisson2d_8192):
    """The same grid in FP32-inner refinement, 2 steps of 50 inner sweeps."""
    p = poisson2d_8192
    period, steps = CHECK_EVERY, 2
    with J.Solver(p.dims, p.block, dtype="f32_refine", faces=p.faces, source=p.source, x0=p.x0,
                  check_every=CHECK_EVERY, refine_period=period, profile=1) as s:
        st, sw, rel = s.solve(1e-300, steps * period)
        field = s.field()
    assert st == J.ERR_NOT_CONVERGED and sw == steps * period
    x0 = p.x0

    def run(d, f, src, xw):
        return oracle.refine_solve(d, f, src, xw, 1e-300, steps * period, period)[1]
    check_samples(p, field, steps * (period + 1) + 1, run, 16, 72)


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False)])
def test_fullsize_3d_512_refine(dtype, e16, r16):
    """512^3, blocks of 64^3, 2 refinement steps of 20 inner sweeps, as the
    3D workload runs (outer step split, inner sweeps with the next line's
    loads issued ahead)."""
    p = inputs.poisson_3d()
    period, steps = 20, 2
    with J.Solver(p.dims, p.block, dtype=dtype, faces=p.faces, source=p.source, x0=p.x0,
                  check_every=CHECK_EVERY, refine_period=period, profile=1) as s:
        st, sw, rel = s.solve(1e-300, steps * period)
        field = s.field()
    assert st == J.ERR_NOT_CONVERGED and sw == steps * period

    def run(d, f, src, xw):
        return oracle.refine_solve(d, f, src, xw, 1e-300, steps * period, period, e_bf16=e16, r_bf16=r16)[1]
    check_samples(p, field, steps * (period + 1) + 1, run, 12, 73)


def test_fullsize_3d_512_f64():
    p = inputs.poisson_3d()
    k = 20
    with J.Solver(p.dims, p.block, dtype="f64", faces=p.faces, source=p.source, x0=p.x0,
                  check_every=CHECK_EVERY, refine_period=CHECK_EVERY, profile=1) as s:
        st, sw, rel = s.solve(1e-300, k)
        field = s.field()
    assert st == J.ERR_NOT_CONVERGED and sw == k
    check_samples(p, field, k, lambda d, f, src, x0: oracle.sweeps(d, f, src, x0, k), 16, 74)


def test_fullsize_batch_256():
    """The full 256-problem batch (sides 64..2048 per axis, 128^2 blocks) with
    the options bench.py uses (persistent schedule, CUDA graphs, autotuner),
    2 refinement steps; sampled points of the largest, the smallest and two
    other problems."""
    probs = inputs.batched_2d(count=256)
    period, steps = 20, 2
    with J.Batch(probs, dtype="f32_refine", refine_period=period, schedule=1, graph=1, autotune=1) as b:
        st, res = b.solve(1e-300, steps * period)
        order = sorted(range(len(probs)), key=lambda i: probs[i].points)
        picks = [order[-1], order[0], order[len(order) // 3], order[2 * len(order) // 3]]
        fields = {i: b.field(i) for i in picks}
    assert all(r[0] == J.ERR_NOT_CONVERGED and r[1] == steps * period for r in res)

    def run(d, f, src, xw):
        return oracle.refine_solve(d, f, src, xw, 1e-300, steps * period, period)[1]
    for i in picks:
        check_samples(probs[i], fields[i], steps * (period + 1) + 1, run, 6, 75 + i)


@pytest.mark.parametrize("form", ["f32_refine", "bf16_refine"])
def test_time_to_tolerance_solves_pass_the_oracle(form):
    """The time-to-tolerance workloads (512^2 in 2D, 128^3 in 3D, to relative
    residual 1e-8, in the options the benchmark times): the oracle recomputes
    the relative residual of each returned field from scratch."""
    for p in (inputs.make_problem((512, 512), (128, 128), 2309, boundary="uniform", source="normal", x0="zero"),
              inputs.poisson_3d(n=128, block=32)):
        with J.Solver(p.dims, p.block, dtype=form, faces=p.faces, source=p.source, check_every=CHECK_EVERY,
                      refine_period=20 if p.ndim == 3 else 50, schedule=1, graph=1, autotune=1) as s:
            st, sw, rel = s.solve(1e-8, 10 ** 9)
            x = s.field()
        assert st == J.OK and rel <= 1e-8
        assert oracle.relative_residual(p.dims, p.faces, p.source, x) <= 1e-8 * (1 + 1e-9)
