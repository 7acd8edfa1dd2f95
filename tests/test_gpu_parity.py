"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Readings (section 4.3's Jacobi proxy): FP64 sweeps in the canonical order
are bit-identical to the oracle (gate: 1e-13 relative per point); the
over-decomposed sweep (section 4.4) is bit-identical to the monolithic one;
refinement solves reach a relative residual <= 1e-8 checked by the oracle.
"""
import json
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


def per_point_close(g, c, rtol=1e-13):
    """|g - c| <= rtol * max(|c|, 1e-3 ||c||_inf) at every point."""
    scale = np.maximum(np.abs(c), 1e-3 * np.max(np.abs(c)) + 1e-300)
    return np.all(np.abs(g - c) <= rtol * scale)


def solver(p, block=None, dtype="f64", **opt):
    return J.Solver(p.dims, block or p.block, dtype=dtype, faces=p.faces, source=p.source, x0=p.x0, **opt)


# ---- plain FP64 sweeps vs the oracle ---------------------------------------

CASES_2D = [
    ((256, 256), (64, 64), 100),
    ((130, 77), (64, 32), 13),       # remainder blocks on both axes
    ((200, 3), (50, 3), 9),
    ((1, 1), (1, 1), 5),             # a single point
    ((1, 40), (1, 7), 6),
    ((65, 1), (64, 1), 4),           # ragged segment tail
    ((129, 70), (129, 70), 11),      # monolithic, odd width
]

CASES_3D = [
    ((37, 29, 23), (16, 8, 8), 12),
    ((64, 64, 64), (64, 64, 64), 3),
    ((20, 6, 9), (7, 5, 2), 7),
    ((3, 1, 2), (1, 1, 1), 4),
    ((130, 9, 5), (64, 4, 3), 5),
]


@pytest.mark.parametrize("dims,block,k", CASES_2D + CASES_3D)
def test_sweeps_match_oracle(dims, block, k):
    p = inputs.make_problem(dims, block, 41, boundary="uniform", source="normal", x0="uniform")
    with solver(p) as s:
        s.sweep(k)
        got = s.field()
    ref = oracle.sweeps(p.dims, p.faces, p.source, p.x0, k)
    assert per_point_close(got, ref)
    assert np.array_equal(got, ref)  # expected: identical operation order


def test_laplace_256_matches_golden_fixture():
    path = os.path.join(os.path.dirname(__file__), "golden", "laplace_2d_256_100.json")
    doc = json.load(open(path))
    p = inputs.laplace_2d_small()
    with solver(p) as s:
        s.sweep(doc["sweeps"])
        x = s.field()
        rel, ab = s.residual()
    for y, xx, v in doc["points"]:
        assert x[y, xx] == float.fromhex(v)
    rss = float.fromhex(doc["rss"])
    assert abs(ab * ab - rss) <= 1e-12 * rss


# ---- over-decomposition invariance (bit-exact) -----------------------------

@pytest.mark.parametrize("dims,blocks", [
    ((300, 190), [(300, 190), (64, 64), (100, 37), (7, 190), (300, 1), (33, 50)]),
    ((40, 33, 27), [(40, 33, 27), (8, 8, 8), (13, 5, 27), (40, 1, 3), (5, 33, 1)]),
])
@pytest.mark.parametrize("halo", [0, 1])
def test_over_decomposition_bit_exact(dims, blocks, halo):
    p = inputs.make_problem(dims, dims, 43, boundary="uniform", source="normal", x0="uniform")
    ref = None
    for b in blocks:
        with solver(p, block=b, halo=halo) as s:
            s.sweep(17)
            x = s.field()
        if ref is None:
            ref = x
        assert np.array_equal(x, ref), b


@pytest.mark.parametrize("rows", [1, 3, 64])
def test_work_item_shape_does_not_change_results(rows):
    p = inputs.make_problem((150, 140), (64, 70), 44, boundary="uniform", source="normal", x0="uniform")
    with solver(p) as s:
        s.sweep(9)
        ref = s.field()
    with solver(p, rows_f64=rows) as s:
        s.sweep(9)
        assert np.array_equal(s.field(), ref)
    p3 = inputs.make_problem((70, 20, 30), (64, 10, 16), 45, boundary="uniform", source="normal", x0="uniform")
    with solver(p3) as s:
        s.sweep(5)
        ref3 = s.field()
    with solver(p3, rows_f64=rows) as s:
        s.sweep(5)
        assert np.array_equal(s.field(), ref3)


# ---- residual ---------------------------------------------------------------

@pytest.mark.parametrize("dims,block", [((256, 200), (64, 64)), ((70, 40, 30), (64, 16, 8)), ((5, 7), (2, 3))])
def test_residual_matches_oracle(dims, block):
    p = inputs.make_problem(dims, block, 46, boundary="uniform", source="normal", x0="uniform")
    with solver(p) as s:
        s.sweep(3)
        x = s.field()
        rel, ab = s.residual()
    rss, bss = oracle.residual(p.dims, p.faces, p.source, x)
    assert abs(ab - np.sqrt(rss)) <= 1e-12 * np.sqrt(rss)
    assert abs(rel - np.sqrt(rss) / np.sqrt(bss)) <= 1e-12 * rel


def test_residual_decomposition_independent():
    """Residual partials are keyed on (group of 8 lines, 64-point segment), so
    any decomposition whose block extents are multiples of 64 along x and of
    8 along the march axis gives the same bits."""
    p = inputs.make_problem((256, 100), (256, 100), 47, boundary="uniform", source="normal", x0="uniform")
    vals = []
    for b in [(256, 100), (64, 8), (128, 32), (64, 96), (192, 40)]:
        with solver(p, block=b) as s:
            s.sweep(4)
            vals.append(s.residual())
    assert all(v == vals[0] for v in vals)


# ---- closed forms on the GPU -------------------------------------------------

def test_gpu_eigenmode_decay():
    from tests.test_oracle_pins import decay_factor, sine_mode
    for dims, modes, block in [((63, 47), (3, 5), (32, 16)), ((19, 17, 15), (2, 1, 3), (8, 8, 4))]:
        x0 = sine_mode(dims, modes)
        lam = decay_factor(dims, modes)
        with J.Solver(dims, block, x0=x0) as s:
            s.sweep(20)
            x = s.field()
        assert np.max(np.abs(x - lam ** 20 * x0)) <= (4 + 8 * 20) * np.finfo(float).eps


def test_gpu_harmonic_fixed_point():
    from tests.test_oracle_pins import field_and_faces, harmonic_fields
    for dims, block in [((31, 17), (8, 8)), ((9, 10, 11), (4, 3, 5))]:
        for u in harmonic_fields(len(dims)):
            inner, faces = field_and_faces(dims, u)
            with J.Solver(dims, block, faces=faces, x0=inner) as s:
                s.sweep(15)
                assert np.array_equal(s.field(), inner)


# ---- solve ---------------------------------------------------------------------

@pytest.mark.parametrize("dims,block", [((48, 40), (16, 16)), ((14, 12, 10), (7, 6, 5))])
def test_solve_f64_matches_oracle(dims, block):
    p = inputs.make_problem(dims, block, 48, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, rel_o = oracle.solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 25)
    with solver(p, check_every=25) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and st_o == oracle.OK
    assert sw == sw_o
    assert np.array_equal(x, x_o)
    assert abs(rel - rel_o) <= 1e-10 * rel_o


def test_solve_cap_and_continue():
    p = inputs.make_problem((40, 30), (20, 10), 49, boundary="uniform", source="normal", x0="zero")
    with solver(p, check_every=7) as s:
        st, sw, rel = s.solve(1e-14, 30)
        assert st == J.ERR_NOT_CONVERGED and sw == 30
        assert J.jacobi_last_error(s.h).startswith("not converged after 30 sweeps")
        x30 = s.field()
        st, sw, rel = s.solve(1e-14, 5)
        assert sw == 5
        x35 = s.field()
    assert np.array_equal(x30, oracle.sweeps(p.dims, p.faces, p.source, None, 30))
    assert np.array_equal(x35, oracle.sweeps(p.dims, p.faces, p.source, None, 35))


# ---- mixed-precision refinement ---------------------------------------------

@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("dims,block", [((60, 45), (32, 16)), ((16, 14, 12), (8, 7, 6)),
                                        # 3D rows narrower than a warp row: 2-16 rows per warp,
                                        # row counts that leave idle lanes, remainder blocks
                                        ((40, 33, 20), (32, 11, 20)), ((70, 9, 8), (64, 5, 4)),
                                        ((130, 6, 7), (130, 6, 7))])
def test_refine_matches_oracle_emulation(dtype, e16, r16, dims, block):
    p = inputs.make_problem(dims, block, 50, boundary="uniform", source="normal", x0="zero")
    period = 20
    st_o, x_o, sw_o, rel_o = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, period,
                                                 e_bf16=e16, r_bf16=r16)
    with solver(p, dtype=dtype, refine_period=period) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and st_o == oracle.OK
    assert oracle.relative_residual(p.dims, p.faces, p.source, x) <= 1e-8
    assert sw == sw_o
    assert np.array_equal(x, x_o)


@pytest.mark.parametrize("halo", [0, 1])
def test_refine_r_bf16_2d_matches_oracle_emulation(halo):
    """e and r both stored as bfloat16, 2D blocks with remainders, the halo of
    e exchanged by the fused push or by the standalone pack/unpack kernels:
    same inner-sweep count and the same field bits as the oracle's emulation,
    and a relative residual <= 1e-8 by the oracle."""
    p = inputs.make_problem((50, 40), (24, 15), 51, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 20,
                                             e_bf16=True, r_bf16=True)
    with solver(p, dtype="bf16r16_refine", refine_period=20, halo=halo) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and st_o == oracle.OK
    assert sw == sw_o
    assert np.array_equal(x, x_o)
    assert oracle.relative_residual(p.dims, p.faces, p.source, x) <= 1e-8


def test_refine_sweep_then_field_is_updated():
    p = inputs.make_problem((64, 64), (32, 32), 52, boundary="uniform", source="normal", x0="uniform")
    with solver(p, dtype="f32_refine", refine_period=10) as s:
        s.sweep(30)
        x = s.field()
    xp = oracle.sweeps(p.dims, p.faces, p.source, p.x0, 30)
    corr = np.max(np.abs(xp - p.x0))
    assert np.max(np.abs(x - xp)) <= 4 * 30 * 2.0 ** -23 * corr


# ---- errors and edge cases ------------------------------------------------------

def test_invalid_arguments():
    with pytest.raises(J.JacobiError) as e:
        J.Solver((10, 10), (11, 10))
    assert e.value.status == J.ERR_INVALID
    with pytest.raises(J.JacobiError):
        J.Solver((10, 10, 10, 10), (1, 1, 1, 1))
    with J.Solver((10, 10), (5, 5)) as s:
        with pytest.raises(J.JacobiError):
            s.set_option("check_every", 0)
        with pytest.raises(J.JacobiError):
            s.set_option("no_such_option", 1)
        # the defaults of the measured forms, and their ranges
        assert s.get_option("march") == 3 and s.get_option("stage3") == 1
        for key, bad in (("march", 4), ("stage3", 2), ("tb", 3), ("march", -1)):
            with pytest.raises(J.JacobiError):
                s.set_option(key, bad)
        assert s.get_option("march") == 3
        st = J.load().jacobi_solve(s.h, -1.0, 10, None, None)
        assert st == J.ERR_INVALID
        s.sweep(0)


def test_set_field_and_source_round_trip():
    p = inputs.make_problem((90, 70), (32, 32), 53, boundary="uniform", source="normal", x0="uniform")
    with solver(p) as s:
        x1 = inputs.uniform(7, 1, 90 * 70).reshape(70, 90)
        s.set_field(x1)
        assert np.array_equal(s.field(), x1)
        f2 = inputs.normal(7, 2, 90 * 70).reshape(70, 90)
        s.set_source(f2)
        s.sweep(6)
        ref = oracle.sweeps(p.dims, p.faces, f2, x1, 6)
        assert np.array_equal(s.field(), ref)
        rel, _ = s.residual()
        assert abs(rel - oracle.relative_residual(p.dims, p.faces, f2, ref)) <= 1e-12 * rel


def test_device_field_io():
    p = inputs.make_problem((64, 48), (32, 16), 54, boundary="uniform", source="normal", x0="uniform")
    with solver(p) as s:
        s.sweep(3)
        out = torch.empty(p.shape, dtype=torch.float64, device="cuda")
        s.field(out)
        torch.cuda.synchronize()
        host = s.field()
        assert np.array_equal(out.cpu().numpy(), host)
        s.set_field(out * 2)
        torch.cuda.synchronize()
        assert np.array_equal(s.field(), host * 2)


@pytest.mark.parametrize("dims,block", [((64, 48), (32, 16)), ((37, 29, 23), (16, 8, 8))])
def test_pinned_host_field_io(dims, block):
    """Page-locked host buffers are read and written by the layout kernels
    directly; the values equal the staged path's (pageable numpy) both ways."""
    p = inputs.make_problem(dims, block, 55, boundary="uniform", source="normal", x0="uniform")
    with solver(p) as s:
        s.sweep(3)
        pinned = torch.empty(p.shape, dtype=torch.float64).pin_memory()
        s.field(pinned)
        pageable = s.field()
        assert np.array_equal(pinned.numpy(), pageable)
        pinned.mul_(3.0)
        s.set_field(pinned)
        pinned.zero_()  # the call returned: the buffer is the caller's again
        assert np.array_equal(s.field(), pageable * 3.0)


def test_two_live_solvers_share_allocator_hooks():
    """Creating a second context must leave the first one usable (the
    allocator hooks a context captured stay valid)."""
    p = inputs.make_problem((64, 40), (32, 20), 55, boundary="uniform", source="normal", x0="uniform")
    a = solver(p)
    b = solver(p, dtype="f32_refine")
    c = solver(p, dtype="bf16_refine")
    a.sweep(4)
    a.set_field(p.x0)
    a.sweep(4)
    xa = a.field()
    b.sweep(4)
    c.sweep(4)
    for s in (c, b, a):
        s.close()
    assert np.array_equal(xa, oracle.sweeps(p.dims, p.faces, p.source, p.x0, 4))


@pytest.mark.parametrize("emu", [2, 3])
@pytest.mark.parametrize("dims,block", [((300, 190), (64, 64)), ((130, 77), (64, 32)), ((37, 29, 23), (16, 8, 8)),
                                        ((65, 1), (64, 1))])
def test_integer_pipe_additions_bit_exact(emu, dims, block):
    """FP64 additions moved to the integer pipe give the same bits."""
    p = inputs.make_problem(dims, block, 56, boundary="uniform", source="normal", x0="uniform")
    with solver(p, emu_adds=emu) as s:
        s.sweep(11)
        got = s.field()
    assert np.array_equal(got, oracle.sweeps(p.dims, p.faces, p.source, p.x0, 11))
    # zeros everywhere (f = 0, g = 0, x = 0) take the fast path's zero rule
    q = inputs.make_problem(dims, block, 57, boundary="zero", source="zero", x0="zero")
    with solver(q, emu_adds=emu) as s:
        s.sweep(3)
        assert not np.any(s.field())


@pytest.mark.parametrize("halo", [0, 1])
@pytest.mark.parametrize("dims,block", [((300, 190), (300, 190)), ((1000, 300), (200, 150)), ((130, 77), (64, 32)),
                                        ((257, 700), (257, 700)), ((37, 29, 23), (16, 8, 8)),
                                        ((200, 9, 150), (130, 9, 150)), ((65, 1), (64, 1)), ((3, 2), (1, 1)),
                                        # 4-point lanes: block widths 1..5 and 127..129 around a segment,
                                        # ragged last lanes, many blocks per row
                                        ((5, 33), (5, 11)), ((129, 40), (129, 40)), ((383, 70), (127, 70)),
                                        ((512, 100), (128, 50)), ((7, 9), (2, 4))])
def test_march_items_bit_exact(halo, dims, block):
    """One warp over all segments of a line range (edge pairs handed on in
    shared memory), with two (march = 1) or four (march = 2, 3) points per
    lane, gives the bits of the per-segment items and of the oracle."""
    p = inputs.make_problem(dims, block, 59, boundary="uniform", source="normal", x0="uniform")
    out = {}
    for march in (0, 1, 2, 3):
        with solver(p, march=march, halo=halo) as s:
            s.sweep(9)
            out[march] = s.field()
    # lines prefetched into L2 ahead of the loads change no bit
    with solver(p, march=2, halo=halo, l2pf=3) as s:
        s.sweep(9)
        out["pf"] = s.field()
    assert np.array_equal(out[1], out[0])
    assert np.array_equal(out[2], out[0])
    assert np.array_equal(out[3], out[0])
    assert np.array_equal(out["pf"], out[0])
    assert np.array_equal(out[1], oracle.sweeps(p.dims, p.faces, p.source, p.x0, 9))


MARCH_R_CASES = [((60, 45), (32, 16)), ((130, 77), (64, 32)), ((5, 33), (5, 11)), ((129, 40), (129, 40)),
                 ((383, 70), (127, 70)), ((512, 100), (128, 50)), ((7, 9), (2, 4)), ((300, 190), (300, 190)),
                 ((65, 1), (64, 1)), ((200, 3), (50, 3)), ((1000, 300), (200, 150))]


@pytest.mark.parametrize("halo", [0, 1])
@pytest.mark.parametrize("dims,block", MARCH_R_CASES)
def test_march_fused_residual_sweep_bit_exact(halo, dims, block):
    """The fused-residual FP64 sweep over march items whose line ranges are
    whole residual groups (four points per lane, lines staged; march = 3)
    writes the field and the residual partials of the per-segment items bit
    for bit: the same status, sweep count, relative residual at every check
    and field as march = 0, and the oracle's solve rule."""
    p = inputs.make_problem(dims, block, 61, boundary="uniform", source="normal", x0="uniform")
    out = {}
    for march in (0, 3):
        with solver(p, march=march, halo=halo, check_every=9) as s:
            st, sw, rel = s.solve(1e-14, 95)
            x1 = s.field()
            st2, sw2, rel2 = s.solve(1e-15, 20)
            out[march] = (st, sw, rel, st2, sw2, rel2, x1, s.field())
    assert out[3][:6] == out[0][:6]
    assert np.array_equal(out[3][6], out[0][6]) and np.array_equal(out[3][7], out[0][7])
    st_o, x_o, sw_o, rel_o = oracle.solve(p.dims, p.faces, p.source, p.x0, 1e-14, 95, 9)
    assert out[3][0] == st_o and out[3][1] == sw_o
    assert abs(out[3][2] - rel_o) <= 1e-10 * rel_o
    assert np.array_equal(out[3][6], x_o)


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("halo", [0, 1])
@pytest.mark.parametrize("dims,block,period", [((60, 45), (32, 16), 20), ((130, 77), (64, 32), 7),
                                               ((5, 33), (5, 11), 10), ((383, 70), (127, 70), 9),
                                               ((7, 9), (2, 4), 5), ((257, 40), (128, 20), 11)])
def test_march_outer_step_bit_exact(dtype, e16, r16, halo, dims, block, period):
    """The refinement's outer step (x_new = x + e, r = b - A x_new stored in
    the low type, residual partials) over residual-aligned march items: the
    same status, inner-sweep count, relative residual and field as the
    per-segment items, and the oracle's emulation."""
    p = inputs.make_problem(dims, block, 62, boundary="uniform", source="normal", x0="zero")
    res = {}
    for march in (0, 3):
        with solver(p, dtype=dtype, refine_period=period, march=march, halo=halo) as s:
            st, sw, rel = s.solve(1e-8, 10 ** 6)
            res[march] = (st, sw, rel, s.field())
    assert res[3][:3] == res[0][:3]
    assert np.array_equal(res[3][3], res[0][3])
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, period,
                                             e_bf16=e16, r_bf16=r16)
    assert res[3][0] == J.OK and st_o == oracle.OK
    assert res[3][1] == sw_o
    assert np.array_equal(res[3][3], x_o)


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("halo", [0, 1])
@pytest.mark.parametrize("dims,block,period", [((40, 33, 20), (32, 11, 20), 20), ((70, 9, 8), (64, 5, 4), 7),
                                               ((16, 14, 12), (8, 7, 6), 10), ((130, 20, 9), (64, 16, 9), 6),
                                               ((5, 6, 7), (1, 1, 1), 5), ((200, 12, 10), (200, 12, 10), 9)])
def test_lane_staged_3d_inner_sweeps_bit_exact(dtype, e16, r16, halo, dims, block, period):
    """3D inner sweeps with each lane's e and r values staged four lines ahead
    in shared memory (stage3 = 1, the default) against one line ahead in
    registers (stage3 = 0) and the oracle's emulation: the same status, sweep
    count and field bits, over rows narrower than a warp, 1-point blocks,
    remainders, both halo modes and all three storage types."""
    p = inputs.make_problem(dims, block, 63, boundary="uniform", source="normal", x0="zero")
    res = {}
    for st3 in (0, 1):
        with solver(p, dtype=dtype, refine_period=period, stage3=st3, halo=halo) as s:
            st, sw, rel = s.solve(1e-8, 10 ** 6)
            res[st3] = (st, sw, rel, s.field())
    assert res[1][:3] == res[0][:3]
    assert np.array_equal(res[1][3], res[0][3])
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, period,
                                             e_bf16=e16, r_bf16=r16)
    assert res[1][0] == J.OK and st_o == oracle.OK
    assert res[1][1] == sw_o
    assert np.array_equal(res[1][3], x_o)


def test_residual_decomposition_independent_3d():
    p = inputs.make_problem((130, 20, 40), (130, 20, 40), 58, boundary="uniform", source="normal", x0="uniform")
    vals = []
    for b in [(130, 20, 40), (64, 7, 8), (128, 20, 16), (64, 3, 24)]:
        with solver(p, block=b) as s:
            s.sweep(3)
            vals.append(s.residual())
    assert all(v == vals[0] for v in vals)


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("dims,block", [((60, 45), (32, 16)), ((300, 70), (130, 33)), ((513, 9), (513, 9)),
                                        ((7, 200), (7, 64)),
                                        # 3D: several rows per warp with idle rows, remainder
                                        # blocks, rows two warp segments wide, one-line items
                                        ((40, 33, 20), (32, 11, 20)), ((70, 9, 8), (64, 5, 4)),
                                        ((300, 4, 5), (300, 4, 5)), ((5, 7, 3), (5, 7, 1))])
def test_staged_inner_sweeps_match_oracle(dtype, e16, r16, dims, block):
    """Inner sweeps with lines staged in shared memory by bulk copies give the
    same bits as the register path and the oracle's emulation."""
    p = inputs.make_problem(dims, block, 59, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 20,
                                             e_bf16=e16, r_bf16=r16)
    with solver(p, dtype=dtype, refine_period=20, tma=1) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and sw == sw_o and np.array_equal(x, x_o)


@pytest.mark.parametrize("dtype", ["f64", "f32_refine"])
def test_checkpoint_and_resume(dtype):
    """A solve interrupted at a check, saved with get_field and resumed in a
    new context from the saved field ends on the same field as one run."""
    p = inputs.make_problem((90, 60), (32, 32), 65, boundary="uniform", source="normal", x0="zero")
    opt = dict(check_every=20, refine_period=20)
    with solver(p, dtype=dtype, **opt) as s:
        st, sw, _ = s.solve(1e-8, 10 ** 6)
        full = s.field()
    with solver(p, dtype=dtype, **opt) as s:
        s.solve(1e-30, 400)
        saved = s.field()
    q = inputs.Problem(p.dims, p.block, p.faces, p.source, saved)
    with solver(q, dtype=dtype, **opt) as s:
        st2, sw2, _ = s.solve(1e-8, 10 ** 6)
        resumed = s.field()
    assert st == st2 == J.OK
    assert sw2 + 400 == sw
    if dtype == "f64":
        assert np.array_equal(resumed, full)
    else:
        # the pending correction is applied at the checkpoint, so the resumed
        # run restarts its inner sweeps from r of the saved field: the same
        # steps, bit for bit
        assert np.array_equal(resumed, full)


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False)])
def test_refine_3d_standalone_halo_matches_oracle(split, dtype, e16, r16):
    """3D refinement with the standalone pack/unpack halo exchange, the outer
    step fused or split, against the oracle's emulation."""
    p = inputs.make_problem((30, 22, 19), (16, 8, 7), 57, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, 20,
                                             e_bf16=e16, r_bf16=r16)
    with solver(p, dtype=dtype, refine_period=20, halo=1, outer_split=split) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and sw == sw_o and np.array_equal(x, x_o)


# ---- two inner sweeps per launch (temporal blocking, 2D) ----------------------

TB_CASES = [((60, 45), (32, 16), 20), ((130, 77), (64, 32), 7), ((5, 33), (1, 11), 10), ((9, 7), (3, 1), 9),
            ((300, 70), (130, 33), 20), ((513, 9), (513, 9), 6), ((257, 40), (128, 20), 11), ((2, 2), (1, 1), 4)]


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("dims,block,period", TB_CASES)
def test_two_sweeps_per_launch_match_oracle_emulation(dtype, e16, r16, dims, block, period):
    """Inner sweeps fused in pairs (the first sweep's values kept in registers,
    neighbour blocks' rows, columns, r and ghost corners read in place): the
    same inner-sweep count and the same field bits as the oracle's emulation
    of single sweeps, over 1-wide and 1-tall blocks, ragged segments,
    remainder blocks and odd refinement periods."""
    p = inputs.make_problem(dims, block, 71, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, period,
                                             e_bf16=e16, r_bf16=r16)
    with solver(p, dtype=dtype, refine_period=period, tb=2) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and st_o == oracle.OK
    assert sw == sw_o
    assert np.array_equal(x, x_o)


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("dims,block", [((200, 150), (64, 48)), ((37, 90), (37, 30))])
def test_two_sweeps_per_launch_equal_single_sweeps(graph, dims, block):
    """jacobi_sweep over several refinement steps (a partial last step too),
    fused pairs against one sweep per launch: identical fields."""
    p = inputs.make_problem(dims, block, 72, boundary="uniform", source="normal", x0="uniform")
    out = {}
    for tb in (0, 2):
        with solver(p, dtype="f32_refine", refine_period=12, tb=tb, graph=graph) as s:
            s.sweep(31)
            out[tb] = s.field()
    assert np.array_equal(out[2], out[0])


TB3_CASES = [((40, 33, 20), (32, 11, 20), 20), ((70, 9, 8), (64, 5, 4), 7), ((16, 14, 12), (8, 7, 6), 10),
             ((130, 20, 9), (64, 16, 9), 6), ((5, 6, 7), (1, 1, 1), 5), ((66, 40, 18), (66, 17, 5), 9),
             # several 16-plane chunks per block, a partial last chunk
             ((24, 20, 40), (24, 20, 40), 8), ((30, 17, 35), (16, 17, 33), 11)]


@pytest.mark.parametrize("dtype,e16,r16", [("f32_refine", False, False), ("bf16_refine", True, False),
                                           ("bf16r16_refine", True, True)])
@pytest.mark.parametrize("dims,block,period", TB3_CASES)
def test_two_sweeps_per_launch_3d_match_oracle_emulation(dtype, e16, r16, dims, block, period):
    """3D inner sweeps fused in pairs (a CTA per (x, y) tile marching along z,
    neighbour planes, rows, columns and the edges of their ghost rings read in
    place): the same inner-sweep count and field bits as the oracle's
    emulation of single sweeps, over ragged and partial tiles, 1x1x1 blocks,
    remainder blocks and odd refinement periods."""
    p = inputs.make_problem(dims, block, 73, boundary="uniform", source="normal", x0="zero")
    st_o, x_o, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, None, 1e-8, 10 ** 6, period,
                                             e_bf16=e16, r_bf16=r16)
    with solver(p, dtype=dtype, refine_period=period, tb=2) as s:
        st, sw, rel = s.solve(1e-8, 10 ** 6)
        x = s.field()
    assert st == J.OK and st_o == oracle.OK
    assert sw == sw_o
    assert np.array_equal(x, x_o)
