"""The dependency-cone windows used by the full-size GPU parity tests agree
with the oracle run on the whole grid (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2303_02543_gb300 import inputs

from cones import sample_points, value_at, window


@pytest.mark.parametrize("dims,block,k", [((300, 200), (128, 64), 20), ((61, 47, 39), (32, 16, 16), 7)])
def test_sweep_windows_match_the_full_run(dims, block, k):
    p = inputs.make_problem(dims, block, 61, boundary="uniform", source="normal", x0="uniform")
    full = oracle.sweeps(p.dims, p.faces, p.source, p.x0, k)
    for c in sample_points(dims, block, 24, 62):
        wd, wf, ws, wx, idx = window(p, c, k)
        got = oracle.sweeps(wd, wf, ws, wx, k)
        assert value_at(got, idx) == value_at(full, c), c


@pytest.mark.parametrize("e16,r16", [(False, False), (True, False)])
def test_refine_windows_match_the_full_run(e16, r16):
    dims, block, period, steps = (45, 40, 38), (16, 16, 16), 5, 2
    p = inputs.make_problem(dims, block, 63, boundary="uniform", source="normal", x0="zero")
    st, full, sw, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-300, steps * period, period,
                                          e_bf16=e16, r_bf16=r16)
    assert sw == steps * period
    radius = steps * (period + 1) + 1
    for c in sample_points(dims, block, 10, 64):
        wd, wf, ws, wx, idx = window(p, c, radius)
        _, got, _, _ = oracle.refine_solve(wd, wf, ws, wx, 1e-300, steps * period, period, e_bf16=e16, r_bf16=r16)
        assert value_at(got, idx) == value_at(full, c), c


def test_too_small_a_window_is_caught():
    """A window short of the cone gives a different value somewhere (so the
    tests above would notice a wrong radius).  The outside values are right
    for the first sweep, so radius k - 1 still suffices; k - 2 does not."""
    dims, block, k = (120, 90), (64, 64), 12
    p = inputs.make_problem(dims, block, 65, boundary="uniform", source="normal", x0="uniform")
    full = oracle.sweeps(p.dims, p.faces, p.source, p.x0, k)
    diffs = 0
    for c in [(60, 45), (30, 50), (90, 20)]:
        wd, wf, ws, wx, idx = window(p, c, k - 2)
        got = oracle.sweeps(wd, wf, ws, wx, k)
        diffs += value_at(got, idx) != value_at(full, c)
    assert diffs > 0
