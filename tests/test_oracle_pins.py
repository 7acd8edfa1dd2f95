"""Pins of the CPU oracle against facts fixed by mathematics, not by itself.

The paper (section 4.3) only says the proxy runs "a fixed number of Jacobi
iterations" on a decomposed 3D domain; the oracle's readings are Poisson with
Dirichlet values, unit spacing, D = 2d I.  Each pin below would fail under a
plausible mistake in the oracle (a dropped neighbour, a wrong divisor or sign,
transposed axes, a missing ghost, a wrong stopping rule).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2303_02543_gb300 import inputs

EPS = np.finfo(np.float64).eps


# ---- pin 1: eigenmode decay (closed form) ----------------------------------

def sin_pi_frac(m, q):
    """sin(pi m / q) for integers, with the argument reduced exactly to
    [0, pi/2] first so that the value is accurate to about one ulp."""
    m = m % (2 * q)
    sign = 1.0
    if m >= q:
        m, sign = m - q, -1.0
    if 2 * m > q:
        m = q - m
    return sign * math.sin(math.pi * m / q)


def sine_mode(dims, modes):
    """Pi_a sin(p_a pi (i_a + 1) / (n_a + 1)) on the interior, x fastest."""
    out = np.ones(tuple(reversed(dims)))
    for a, (n, p) in enumerate(zip(dims, modes)):
        v = np.array([sin_pi_frac(p * i, n + 1) for i in range(1, n + 1)])
        shape = [1] * len(dims)
        shape[len(dims) - 1 - a] = n
        out = out * v.reshape(shape)
    return out


def decay_factor(dims, modes):
    """lambda = (1/d) sum_a cos(p_a pi / (n_a + 1)) (cos(p pi/(n+1)) in 1D)."""
    return sum(math.cos(p * math.pi / (n + 1)) for n, p in zip(dims, modes)) / len(dims)


EIGEN_CASES = [
    ((17,), (1,)),
    ((17,), (17,)),            # highest mode: lambda < 0, sign flips each sweep
    ((16,), (5,)),
    ((23, 17), (1, 1)),
    ((23, 17), (23, 17)),
    ((23, 17), (3, 5)),        # mixed, rectangular: catches swapped axes
    ((40, 9), (7, 2)),
    ((9, 7, 5), (1, 1, 1)),
    ((9, 7, 5), (2, 3, 1)),
    ((9, 7, 5), (9, 7, 5)),
    ((6, 11, 4), (1, 4, 3)),
]


@pytest.mark.parametrize("dims,modes", EIGEN_CASES)
@pytest.mark.parametrize("k", [1, 7, 40])
def test_eigenmode_decay(dims, modes, k):
    x0 = sine_mode(dims, modes)
    lam = decay_factor(dims, modes)
    xk = oracle.sweeps(dims, None, None, x0, k)
    err = np.max(np.abs(xk - lam ** k * x0))
    assert err <= (4 + 8 * k) * EPS * np.max(np.abs(x0)), (err, lam)


def test_eigenmode_decay_distinguishes_axes():
    """A mode that is not symmetric in x and y decays at a rate that changes
    when the axes are swapped; the oracle must follow the right one."""
    dims, modes = (23, 17), (3, 5)
    wrong = decay_factor(dims, (5, 3))
    xk = oracle.sweeps(dims, None, None, sine_mode(dims, modes), 10)
    assert np.max(np.abs(xk - wrong ** 10 * sine_mode(dims, modes))) > 1e-3


# ---- pin 2: discrete-harmonic fixed points (bit-exact) ----------------------

def harmonic_fields(nd):
    if nd == 1:
        return [lambda i: 3 + 5 * i, lambda i: -7 * i + 11]
    if nd == 2:
        return [lambda i, j: 3 + 5 * i - 2 * j, lambda i, j: i * j, lambda i, j: i * i - j * j,
                lambda i, j: 7 * i * j - 3 * i + 4 * j + 1]
    return [lambda i, j, k: 3 + 5 * i - 2 * j + 7 * k, lambda i, j, k: i * j * k,
            lambda i, j, k: i * j + j * k - 2 * i * k, lambda i, j, k: i * i - k * k + 3 * j]


def field_and_faces(dims, u):
    """u on the interior (dense) and on the ghost ring (faces)."""
    nd = len(dims)
    rng = [np.arange(n) for n in dims]
    if nd == 1:
        inner = np.array([u(i) for i in rng[0]], dtype=np.float64)
        return inner, [np.array([u(-1)], float), np.array([u(dims[0])], float)]
    if nd == 2:
        nx, ny = dims
        inner = np.array([[u(i, j) for i in range(nx)] for j in range(ny)], dtype=np.float64)
        faces = [np.array([u(-1, j) for j in range(ny)], float), np.array([u(nx, j) for j in range(ny)], float),
                 np.array([u(i, -1) for i in range(nx)], float), np.array([u(i, ny) for i in range(nx)], float)]
        return inner, faces
    nx, ny, nz = dims
    inner = np.array([[[u(i, j, k) for i in range(nx)] for j in range(ny)] for k in range(nz)], dtype=np.float64)
    faces = [np.array([u(-1, j, k) for k in range(nz) for j in range(ny)], float),
             np.array([u(nx, j, k) for k in range(nz) for j in range(ny)], float),
             np.array([u(i, -1, k) for k in range(nz) for i in range(nx)], float),
             np.array([u(i, ny, k) for k in range(nz) for i in range(nx)], float),
             np.array([u(i, j, -1) for j in range(ny) for i in range(nx)], float),
             np.array([u(i, j, nz) for j in range(ny) for i in range(nx)], float)]
    return inner, faces


@pytest.mark.parametrize("dims", [(13,), (11, 7), (5, 6, 7)])
def test_harmonic_fixed_point_bit_exact(dims):
    for u in harmonic_fields(len(dims)):
        inner, faces = field_and_faces(dims, u)
        out = oracle.sweeps(dims, faces, None, inner, 25)
        assert np.array_equal(out, inner)
        rss, _ = oracle.residual(dims, faces, None, inner)
        assert rss == 0.0


@pytest.mark.parametrize("dims", [(11, 7), (5, 6, 7)])
def test_harmonic_attracts_random_start(dims):
    u = harmonic_fields(len(dims))[1]
    inner, faces = field_and_faces(dims, u)
    x0 = inputs.uniform(5, 1, inner.size).reshape(inner.shape) * 50
    st, x, sw, rel = oracle.solve(dims, faces, None, x0, 1e-12, 200000, 10)
    assert st == oracle.OK and rel <= 1e-12
    assert np.max(np.abs(x - inner)) <= 1e-9 * np.max(np.abs(inner))


# ---- pin 3: manufactured solution (exact integer arithmetic) ----------------

def manufactured(dims, seed):
    """Random integer u* on the grid including its ghost ring; f = A u* and
    the ghost values are computed exactly in int64."""
    nd = len(dims)
    rng = np.random.default_rng(seed)
    ext = rng.integers(-1000, 1000, size=tuple(n + 2 for n in reversed(dims))).astype(np.int64)
    core = tuple(slice(1, -1) for _ in range(nd))
    u = ext[core]
    au = 2 * nd * u
    for ax in range(nd):
        lo = [slice(1, -1)] * nd
        hi = [slice(1, -1)] * nd
        lo[ax] = slice(0, -2)
        hi[ax] = slice(2, None)
        au = au - ext[tuple(lo)] - ext[tuple(hi)]
    # faces from the ghost ring, ordered -x,+x,-y,+y,-z,+z, lowest axis fastest
    faces = []
    for axis in range(nd):
        ax = nd - 1 - axis
        for side in (0, -1):
            sl = [slice(1, -1)] * nd
            sl[ax] = side
            faces.append(ext[tuple(sl)].astype(np.float64).reshape(-1))
    return u.astype(np.float64), faces, au.astype(np.float64)


@pytest.mark.parametrize("dims", [(9,), (12, 9), (6, 5, 7)])
def test_manufactured_solution_exact(dims):
    u, faces, f = manufactured(dims, 17)
    rss, bss = oracle.residual(dims, faces, f, u)
    assert rss == 0.0 and bss > 0
    assert np.array_equal(oracle.sweeps(dims, faces, f, u, 9), u)
    st, x, sw, rel = oracle.solve(dims, faces, f, None, 1e-11, 500000, 25)
    assert st == oracle.OK
    assert np.max(np.abs(x - u)) <= 1e-7 * np.max(np.abs(u))


# ---- pin 4: dense brute force on tiny grids --------------------------------

TINY = [(6,), (5, 4), (7, 6), (3, 4, 5), (4, 3, 2)]


def tiny_problem(dims, seed):
    p = inputs.make_problem(dims, dims, seed, boundary="uniform", source="normal", x0="uniform")
    return p.faces, p.source, p.x0


@pytest.mark.parametrize("dims", TINY)
def test_dense_iteration_matches(dims):
    faces, f, x0 = tiny_problem(dims, 3)
    A, b = dense.assemble(dims, faces, f)
    for k in (1, 5, 30):
        ref = dense.jacobi_matrix_form(A, b, x0, k)
        got = oracle.sweeps(dims, faces, f, x0, k).reshape(-1)
        scale = np.max(np.abs(ref)) + np.max(np.abs(b))
        assert np.max(np.abs(got - ref)) <= 16 * k * EPS * scale


@pytest.mark.parametrize("dims", TINY)
def test_dense_residual_matches(dims):
    faces, f, x0 = tiny_problem(dims, 4)
    A, b = dense.assemble(dims, faces, f)
    rss, bss, r = oracle.residual(dims, faces, f, x0, want_r=True)
    rd = b - A @ x0.reshape(-1)
    assert np.max(np.abs(r.reshape(-1) - rd)) <= 64 * EPS * (np.max(np.abs(b)) + 8 * np.max(np.abs(x0)))
    assert abs(rss - rd @ rd) <= 1e-13 * (rd @ rd)
    assert abs(bss - b @ b) <= 1e-13 * (b @ b)


@pytest.mark.parametrize("dims", TINY)
def test_dense_solution_matches(dims):
    faces, f, x0 = tiny_problem(dims, 5)
    A, b = dense.assemble(dims, faces, f)
    xs = np.linalg.solve(A, b)
    st, x, sw, rel = oracle.solve(dims, faces, f, x0, 1e-13, 10 ** 6, 7)
    assert st == oracle.OK
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x.reshape(-1) - xs) <= 4 * cond * 1e-13 * np.linalg.norm(xs)


@pytest.mark.parametrize("dims", TINY)
def test_spectral_radius_is_mean_of_cosines(dims):
    A, _ = dense.assemble(dims, None, None)
    rho = dense.iteration_spectral_radius(A)
    closed = decay_factor(dims, (1,) * len(dims))
    assert abs(rho - closed) <= 1e-12


# ---- solve semantics --------------------------------------------------------

def test_solve_stops_at_first_checked_iterate():
    p = inputs.make_problem((20, 14), (20, 14), 8, boundary="uniform", source="normal", x0="uniform")
    c = 13
    st, x, sw, rel = oracle.solve(p.dims, p.faces, p.source, p.x0, 1e-6, 10 ** 6, c)
    assert st == oracle.OK and sw % c == 0 and sw > 0 and rel <= 1e-6
    before = oracle.sweeps(p.dims, p.faces, p.source, p.x0, sw - c)
    assert oracle.relative_residual(p.dims, p.faces, p.source, before) > 1e-6
    assert np.array_equal(oracle.sweeps(p.dims, p.faces, p.source, p.x0, sw), x)
    st2, _, sw2, _ = oracle.solve(p.dims, p.faces, p.source, p.x0, 1e-30, 40, c)
    assert st2 == oracle.NOT_CONVERGED and sw2 == 40


def test_zero_rhs_uses_absolute_residual():
    dims = (9, 8)
    x0 = inputs.uniform(1, 1, 72).reshape(8, 9)
    st, x, sw, rel = oracle.solve(dims, None, None, x0, 1e-9, 10 ** 6, 10)
    assert st == oracle.OK
    rss, bss = oracle.residual(dims, None, None, x)
    assert bss == 0.0 and math.sqrt(rss) <= 1e-9


def test_threads_do_not_change_results():
    p = inputs.make_problem((33, 21, 9), (33, 21, 9), 9, boundary="uniform", source="normal", x0="uniform")
    a = oracle.sweeps(p.dims, p.faces, p.source, p.x0, 12, threads=1)
    b = oracle.sweeps(p.dims, p.faces, p.source, p.x0, 12, threads=4)
    assert np.array_equal(a, b)
    assert oracle.residual(p.dims, p.faces, p.source, a, threads=1) == \
        oracle.residual(p.dims, p.faces, p.source, a, threads=4)


# ---- pin 5: bfloat16 rounding and the mixed-precision refinement ------------

def test_round_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    bits = inputs.u64_stream(11, 1, 20000).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    vals = bits.astype(np.uint32).view(np.float32)
    vals = vals[np.isfinite(vals)]
    # exact ties: low half 0x8000 with even and odd kept bits
    ties = (np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40490000 | 0x8000], dtype=np.uint32)).view(np.float32)
    vals = np.concatenate([vals, ties, np.float32([1.0, -2.5, 3.0e38, 1e-40])])
    ref = torch.from_numpy(vals.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.round_bf16(float(v)) for v in vals], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("dims", [(20, 14), (9, 8, 7)])
@pytest.mark.parametrize("e_bf16", [False, True])
def test_refine_step_equals_plain_sweeps_in_exact_arithmetic(dims, e_bf16):
    """k inner sweeps on A e = r from e = 0, then x += e, equal k plain sweeps
    from x in exact arithmetic; in float/bfloat16 they agree to the inner
    precision times the size of the correction."""
    p = inputs.make_problem(dims, dims, 12, boundary="uniform", source="normal", x0="uniform")
    k = 9
    st, xr, sw, _ = oracle.refine_solve(p.dims, p.faces, p.source, p.x0, 1e-300, k, k, e_bf16=e_bf16)
    assert st == oracle.NOT_CONVERGED and sw == k
    xp = oracle.sweeps(p.dims, p.faces, p.source, p.x0, k)
    corr = np.max(np.abs(xp - p.x0))
    unit = 2.0 ** -8 if e_bf16 else 2.0 ** -23
    assert np.max(np.abs(xr - xp)) <= 4 * k * unit * corr
    assert np.max(np.abs(xr - xp)) > 0      # low precision really is in use


@pytest.mark.parametrize("e_bf16,r_bf16", [(False, False), (True, False), (True, True)])
def test_refine_converges_like_fp64(e_bf16, r_bf16):
    p = inputs.make_problem((40, 31), (40, 31), 13, boundary="uniform", source="normal", x0="zero")
    tol = 1e-8
    st64, x64, sw64, _ = oracle.solve(p.dims, p.faces, p.source, None, tol, 10 ** 6, 20)
    st, x, sw, rel = oracle.refine_solve(p.dims, p.faces, p.source, None, tol, 10 ** 6, 20,
                                         e_bf16=e_bf16, r_bf16=r_bf16)
    assert st64 == oracle.OK and st == oracle.OK
    assert oracle.relative_residual(p.dims, p.faces, p.source, x) <= tol
    assert abs(sw - sw64) <= 0.1 * sw64 + 40
    assert np.linalg.norm(x - x64) <= 1e-6 * np.linalg.norm(x64)


@pytest.mark.parametrize("e_bf16,r_bf16", [(False, False), (True, False), (True, True)])
@pytest.mark.parametrize("dims", [(9, 7), (5, 4, 6)])
def test_refinement_reaches_fp64_accuracy_below_the_inner_precision(dims, e_bf16, r_bf16):
    """With the residual and the update x += e in FP64, refinement keeps
    converging after the correction falls below the inner type's precision
    (float 2^-24, bfloat16 2^-9 relative): it reaches rel 1e-13, and x agrees
    with the direct solve of the dense system to cond(A) * 1e-13, as plain
    FP64 Jacobi does.  An update or residual kept in the inner type would
    stall near its precision instead."""
    faces, f, _ = tiny_problem(dims, 6)
    A, b = dense.assemble(dims, faces, f)
    xs = np.linalg.solve(A, b)
    st, x, sw, rel = oracle.refine_solve(dims, faces, f, None, 1e-13, 10 ** 5, 10, e_bf16=e_bf16, r_bf16=r_bf16)
    assert st == oracle.OK and rel <= 1e-13
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x.reshape(-1) - xs) <= 4 * cond * 1e-13 * np.linalg.norm(xs)


def test_refine_from_exact_solution_stops_at_once():
    u, faces, f = manufactured((12, 9), 21)
    st, x, sw, rel = oracle.refine_solve((12, 9), faces, f, u, 1e-12, 100, 10)
    assert st == oracle.OK and sw == 0 and rel == 0.0 and np.array_equal(x, u)


# ---- stored fixture stays reproducible --------------------------------------

def test_golden_fixture_reproduces():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "laplace_2d_256_100.json")
    doc = json.load(open(path))
    p = inputs.laplace_2d_small()
    x = oracle.sweeps(p.dims, p.faces, p.source, p.x0, doc["sweeps"])
    for y, xx, v in doc["points"]:
        assert x[y, xx] == float.fromhex(v)
    rss, bss = oracle.residual(p.dims, p.faces, p.source, x)
    assert rss == float.fromhex(doc["rss"]) and bss == float.fromhex(doc["bss"])


@pytest.mark.parametrize("dims", [(12, 9), (6, 5, 4)])
def test_non_finite_inputs_stop_the_solve_as_diverged(dims):
    """The solve rule on a non-finite residual: a NaN in the source (so ||b||
    and the residual are NaN) or an infinite initial value (an infinite
    residual) stops the plain and the refinement solve at the first test,
    after 0 sweeps, with JO_DIVERGED -- never as converged or capped.  So does
    a NaN in one Dirichlet face value (it enters b)."""
    p = inputs.make_problem(dims, dims, 14, boundary="uniform", source="normal", x0="uniform")
    f_nan = p.source.copy()
    f_nan.flat[f_nan.size // 2] = np.nan
    x_inf = p.x0.copy()
    x_inf.flat[1] = np.inf
    for f, x0 in ((f_nan, p.x0), (p.source, x_inf)):
        st, _, sw, rel = oracle.solve(p.dims, p.faces, f, x0, 1e-8, 100, 10)
        assert st == oracle.DIVERGED and sw == 0 and not np.isfinite(rel)
        st, _, sw, rel = oracle.refine_solve(p.dims, p.faces, f, x0, 1e-8, 100, 10)
        assert st == oracle.DIVERGED and sw == 0 and not np.isfinite(rel)
    faces = [g.copy() for g in p.faces]
    faces[3].flat[0] = np.nan
    st, _, sw, rel = oracle.solve(p.dims, faces, p.source, p.x0, 1e-8, 100, 10)
    assert st == oracle.DIVERGED and sw == 0 and not np.isfinite(rel)
    # the finite problem itself converges (the rule is not triggered by accident)
    st, _, _, rel = oracle.solve(p.dims, p.faces, p.source, p.x0, 1e-3, 10 ** 5, 10)
    assert st == oracle.OK and rel <= 1e-3
