"""Pin strength: plausible mistakes planted in a COPY of the oracle source (on
the CPU) must each be caught by at least one of the pins in
test_oracle_pins.py.  The shipped oracle is never modified."""
import os

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = {
    # a dropped neighbour in the 2D/3D sum
    "drop_north": ("(a[p + G->s[0]] + a[p + sl])", "(a[p + G->s[0]] + 0.0)"),
    # a wrong sign on one neighbour
    "sign_east": ("(a[p + G->s[0]] + a[p + sl])", "(-a[p + G->s[0]] + a[p + sl])"),
    # wrong divisor (d instead of 2d)
    "divisor": ("dst[p] = neighbour_sum_plus_f(G, src, p, fp) / two_d;",
                "dst[p] = neighbour_sum_plus_f(G, src, p, fp) / (two_d - 1.0);"),
    # transposed index in the y neighbour (x stride used twice)
    "transposed": ("s = (a[p - G->s[0]] + a[p - sl])", "s = (a[p - G->s[0]] + a[p - G->s[0]])"),
    # 3D: the y pair replaced by a second z pair
    "axis3d": ("if (G->ndim == 3) s = s + (a[p - G->s[1]] + a[p + G->s[1]]);", "if (G->ndim == 3) s = s + (a[p - G->s[2]] + a[p + G->s[2]]);"),
    # source term dropped from the update
    "no_source": ("  return s + fp;", "  return s + 0.0 * fp;"),
    # residual with the wrong sign on the diagonal term
    "residual_sign": ("- two_d * a[p];", "+ two_d * a[p];"),
    # +y face read from the -y face array
    "face_swap": ("faces[3][i + nx * k]", "faces[2][i + nx * k]"),
    # a stopping rule that tests before the update but returns one check late
    "solve_cadence": ("    m += k;\n  }\n  store_interior(&G, a, x);\n  if (sweeps_out) *sweeps_out = m;",
                      "    m += k + 1;\n  }\n  store_interior(&G, a, x);\n  if (sweeps_out) *sweeps_out = m;"),
    # refinement that forgets to add the correction
    "refine_no_update": ("a[p] = a[p] + (double)e[p];", "a[p] = a[p] + 0.0 * (double)e[p];"),
    # refinement whose update x += e is kept in float
    "refine_float_update": ("a[p] = a[p] + (double)e[p];", "a[p] = (double)(float)(a[p] + (double)e[p]);"),
    # inner sweep of the correction with a wrong sign on one neighbour
    "sweep_low_sign": ("(src[p + G->s[0]] + src[p + sl])", "(-src[p + G->s[0]] + src[p + sl])"),
    # inner sweep that drops its right-hand side r
    "sweep_low_no_rhs": ("const float t = s + r[didx(G, i, j, k)];", "const float t = s + 0.0f * r[didx(G, i, j, k)];"),
    # inner sweep divided by 2d + 1 (a damped iteration with the wrong fixed point)
    "sweep_low_divisor": ("const float v = t / two_d;", "const float v = t / (two_d + 1.0f);"),
}


def run_pins():
    """Run a fixed subset of the pins; return the names that failed."""
    failed = []
    checks = {
        "eigen2d": lambda: pins.test_eigenmode_decay((23, 17), (3, 5), 7),
        "eigen3d": lambda: pins.test_eigenmode_decay((9, 7, 5), (2, 3, 1), 7),
        "harmonic2d": lambda: pins.test_harmonic_fixed_point_bit_exact((11, 7)),
        "manufactured": lambda: pins.test_manufactured_solution_exact((12, 9)),
        "dense_iter": lambda: pins.test_dense_iteration_matches((7, 6)),
        "dense_res": lambda: pins.test_dense_residual_matches((7, 6)),
        "solve_rule": lambda: pins.test_solve_stops_at_first_checked_iterate(),
        "refine": lambda: pins.test_refine_converges_like_fp64(False, False),
        "refine_deep": lambda: pins.test_refinement_reaches_fp64_accuracy_below_the_inner_precision((9, 7), False, False),
        "refine_step": lambda: pins.test_refine_step_equals_plain_sweeps_in_exact_arithmetic((20, 14), False),
    }
    for name, fn in checks.items():
        try:
            fn()
        except Exception:  # noqa: BLE001 - any failure of a pin counts
            failed.append(name)
    return failed


def test_unmutated_copy_passes(tmp_path):
    path = oracle.compile_source(oracle.source_text(), str(tmp_path / "clean.so"))
    with oracle.use_library(path):
        assert run_pins() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert old in src, f"mutation site for {name} not found"
    path = oracle.compile_source(src.replace(old, new, 1), str(tmp_path / f"{name}.so"))
    with oracle.use_library(path):
        failed = run_pins()
    assert failed, f"no pin caught mutant {name}"
