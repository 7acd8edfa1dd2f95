"""CPU-only checks of the CUDA library's host side: it builds, loads and exports
every entry point that include/jacobi.h declares (no compute calls without a
GPU), and the exact FP64 scalings used by the kernels agree bit for bit with
IEEE division."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "jacobi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(jacobi_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_expected_entry_points():
    from paper_2303_02543_gb300 import jacobi as J
    assert declared_symbols() == sorted(J.EXPORTS)


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2303_02543_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(jacobi_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    import ctypes
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert getattr(lib, s) is not None
    lib.jacobi_version.restype = ctypes.c_int
    assert lib.jacobi_version() >= 10000


def test_invalid_arguments_rejected_without_gpu():
    """Argument validation happens before any CUDA call."""
    import ctypes
    from paper_2303_02543_gb300 import build
    from paper_2303_02543_gb300 import jacobi as J
    build.build()
    lib = J.load()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(10, 10, 1)
    bad = (ctypes.c_int64 * 3)(11, 10, 1)
    assert lib.jacobi_create(ctypes.byref(h), 2, dims, bad, 0, None, None, None, None) == J.ERR_INVALID
    assert not h.value
    assert lib.jacobi_create(ctypes.byref(h), 4, dims, dims, 0, None, None, None, None) == J.ERR_INVALID
    assert lib.jacobi_create(ctypes.byref(h), 2, dims, dims, 9, None, None, None, None) == J.ERR_INVALID
    assert b"block" in lib.jacobi_last_error(None) or b"dtype" in lib.jacobi_last_error(None)
    assert lib.jacobi_sweep(None, 1) == J.ERR_INVALID
    lib.jacobi_destroy(None)


def test_exact_f64_helpers_match_ieee(tmp_path):
    src = os.path.join(ROOT, "tests", "native", "exact_f64_check.cpp")
    exe = str(tmp_path / "exact_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2303_02543_gb300", "csrc"),
                    "-o", exe, src], check=True)
    r = subprocess.run([exe, "3000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout


def test_serving_arena_first_fit_matches_brute_force(tmp_path):
    """The serving arena's placement (first_fit.h, host-only C++) against a
    granule-by-granule first-fit model over random allocation and release
    sequences."""
    src = os.path.join(ROOT, "tests", "native", "first_fit_check.cpp")
    exe = str(tmp_path / "first_fit_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2303_02543_gb300", "csrc"), "-o", exe, src], check=True)
    r = subprocess.run([exe, "200000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout


def test_march_runs_dealt_to_warps_meet_their_contract(tmp_path):
    """The dealing of block lines to warps in equal runs (deal_runs.h,
    host-only C++; the 2D FP64 march items) on random block lists: every line
    covered once in block order, pieces inside one block on step boundaries,
    the stated warp count, runs equal to within one step and never longer than
    a warp's shared pair buffer."""
    src = os.path.join(ROOT, "tests", "native", "deal_runs_check.cpp")
    exe = str(tmp_path / "deal_runs_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2303_02543_gb300", "csrc"), "-o", exe, src], check=True)
    r = subprocess.run([exe, "20000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout


def test_one_rounding_residual_equals_the_oracles_subtraction():
    """The kernels form the 2D residual t - 4x as one fused multiply-add,
    RN(t - 4x); the oracle subtracts the product, RN(t - RN(4x)).  4x is exact
    wherever it is finite, so the two agree: checked here on random doubles of
    every magnitude, with the exact difference rounded once (Fraction -> float
    rounds to nearest-even), against the double arithmetic of the oracle."""
    from fractions import Fraction
    rng = np.random.default_rng(2312)
    for _ in range(20000):
        x = float(rng.standard_normal() * 2.0 ** int(rng.integers(-300, 300)))
        t = float(rng.standard_normal() * 2.0 ** int(rng.integers(-300, 300)))
        if rng.random() < 0.3:
            t = 4.0 * x * (1.0 + float(rng.standard_normal()) * 2.0 ** -int(rng.integers(1, 60)))  # cancellation
        one_rounding = float(Fraction(t) - 4 * Fraction(x))
        assert one_rounding == t - 4.0 * x
    # with 6 (3D) the product is not exact and one rounding differs from two,
    # which is why the 3D kernels round 6x first and then fma(6x, -1, t)
    diff = 0
    for _ in range(20000):
        x = float(rng.standard_normal())
        t = 6.0 * x * (1.0 + float(rng.standard_normal()) * 2.0 ** -int(rng.integers(1, 40)))
        diff += float(Fraction(t) - 6 * Fraction(x)) != t - 6.0 * x
    assert diff > 0


def test_torch_allocator_trampolines_are_created_once():
    """A context keeps the allocator hooks it was created with; reinstalling
    must not free the ctypes trampolines those hooks point to."""
    pytest.importorskip("torch")
    from paper_2303_02543_gb300 import build
    from paper_2303_02543_gb300 import jacobi as J
    build.build()
    J.use_torch_allocator(True)
    a, f = J._alloc_cb, J._free_cb
    J.use_torch_allocator(True)
    J.use_torch_allocator(False)
    J.use_torch_allocator(True)
    assert J._alloc_cb is a and J._free_cb is f


@pytest.mark.parametrize("compiler,flags", [("gcc", ["-std=c99", "-x", "c"]), ("g++", ["-std=c++11", "-x", "c++"])])
def test_header_compiles_as_plain_c_and_cpp(tmp_path, compiler, flags):
    """include/jacobi.h is a self-contained C header (usable from C and C++
    without CUDA or torch headers), with no warnings under -pedantic."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not available")
    src = tmp_path / "use_header.c"
    src.write_text('#include "jacobi.h"\n'
                   "int main(void) {\n"
                   "  jacobi_t ctx = 0;\n"
                   "  jacobi_boundary bc;\n"
                   "  (void)ctx; (void)bc;\n"
                   "  return (int)JACOBI_OK;\n"
                   "}\n")
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([compiler, *flags, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, "-c", str(src),
                        "-o", str(tmp_path / "use_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_refuses_field_buffers_of_the_wrong_size_type_or_layout():
    """The C side trusts a field buffer's size, so the binding checks it."""
    import numpy as np
    import torch
    from paper_2303_02543_gb300 import jacobi as J
    shape = (6, 5)
    p, dev = J._ptr(np.zeros(shape), shape, writable=True)
    assert p.value is not None and dev == 0
    p, dev = J._ptr(torch.zeros(shape, dtype=torch.float64), shape)
    assert dev == 0
    bad = [np.zeros(shape, dtype=np.float32), np.zeros((6, 4)), np.zeros((5, 6)).T, [0.0] * 30,
           torch.zeros(shape, dtype=torch.float32), torch.zeros((5, 6), dtype=torch.float64).t(),
           torch.zeros((31,), dtype=torch.float64)]
    for a in bad:
        with pytest.raises(ValueError):
            J._ptr(a, shape)
    ro = np.zeros(shape)
    ro.flags.writeable = False
    J._ptr(ro, shape)
    with pytest.raises(ValueError):
        J._ptr(ro, shape, writable=True)


def test_binding_checks_host_input_sizes_against_the_grid():
    """Source, initial field and Dirichlet faces are read by the C side for
    exactly the grid's sizes; the binding refuses anything else."""
    import numpy as np
    from paper_2303_02543_gb300 import inputs
    from paper_2303_02543_gb300 import jacobi as J
    assert J.face_sizes((7, 5)) == [5, 5, 7, 7]
    assert J.face_sizes((7, 5, 3)) == [15, 15, 21, 21, 35, 35]
    for dims in ((7, 5), (7, 5, 3)):
        p = inputs.make_problem(dims, dims, 3, boundary="random", source="normal", x0="uniform")
        keep = []
        ps = J._problem_struct(p, keep)          # the generator's own shapes pass
        assert ps.ndim == len(dims) and ps.bc.kind == J.BC_FACES
        for q in range(2 * len(dims)):
            faces = list(p.faces)
            faces[q] = np.zeros(faces[q].size + 1)
            with pytest.raises(ValueError):
                J.make_boundary(faces, dims=dims)
        with pytest.raises(ValueError):
            J.make_boundary(list(p.faces) + [np.zeros(1)] * (7 - len(p.faces)), dims=dims)
        for name in ("source", "x0"):
            q = inputs.make_problem(dims, dims, 3, boundary="random", source="normal", x0="uniform")
            setattr(q, name, np.zeros(int(np.prod(dims)) - 1))
            with pytest.raises(ValueError):
                J._problem_struct(q, [])


def test_size_limits_and_empty_inputs_rejected_without_gpu():
    """Empty grids, dimensions of 2^30 and beyond, more than 2^28 blocks, empty
    or oversized batches, and out-of-range server settings are refused with
    JACOBI_ERR_INVALID before any CUDA call (so also on a host without a GPU)."""
    import ctypes
    from paper_2303_02543_gb300 import build
    from paper_2303_02543_gb300 import jacobi as J
    build.build()
    lib = J.load()
    h = ctypes.c_void_p()
    d3 = lambda *v: (ctypes.c_int64 * 3)(*v)  # noqa: E731
    cases = [
        (2, d3(0, 10, 1), d3(1, 1, 1)),                  # empty along x
        (3, d3(10, 10, 0), d3(1, 1, 1)),                 # empty along z
        (2, d3(1 << 30, 1, 1), d3(1 << 20, 1, 1)),       # dimension too large
        (2, d3(1 << 29, 4, 1), d3(1, 1, 1)),             # 2^31 blocks
        (3, d3(1 << 10, 1 << 10, 1 << 9), d3(1, 1, 2)),  # 2^28 blocks exactly
        (2, d3(10, 10, 1), d3(0, 5, 1)),                 # empty block
    ]
    for nd, dims, blk in cases:
        assert lib.jacobi_create(ctypes.byref(h), nd, dims, blk, 0, None, None, None, None) == J.ERR_INVALID
        assert not h.value
    assert lib.jacobi_batch_create(ctypes.byref(h), 0, None, 1, None) == J.ERR_INVALID
    probs = (J.Problem * 1)()
    assert lib.jacobi_batch_create(ctypes.byref(h), (1 << 20) + 1, probs, 1, None) == J.ERR_INVALID
    assert lib.jacobi_batch_create(ctypes.byref(h), 1, probs, 1, None) == J.ERR_INVALID  # ndim 0
    s = ctypes.c_void_p()
    assert lib.jacobi_server_create(ctypes.byref(s), 0, 64 << 20, 4, None) == J.ERR_INVALID   # FP64 is not served
    assert lib.jacobi_server_create(ctypes.byref(s), 1, (1 << 20) - 1, 4, None) == J.ERR_INVALID
    assert lib.jacobi_server_create(ctypes.byref(s), 1, 64 << 20, 0, None) == J.ERR_INVALID
    assert lib.jacobi_server_create(ctypes.byref(s), 1, 64 << 20, 4097, None) == J.ERR_INVALID
    assert not s.value
    x = ctypes.c_void_p(8)  # never dereferenced: validation fails first
    assert lib.jacobi_residual_noalloc(2, d3(0, 4, 1), x, None, None, x, None) == J.ERR_INVALID
    assert lib.jacobi_residual_noalloc(4, d3(4, 4, 4), x, None, None, x, None) == J.ERR_INVALID
    assert lib.jacobi_residual_noalloc(2, d3(1 << 30, 4, 1), x, None, None, x, None) == J.ERR_INVALID
    # beyond the fixed scratch: ceil(nx/64) * ceil(ny/8) partials > 2^20
    assert lib.jacobi_residual_noalloc(2, d3(1 << 16, 1 << 15, 1), x, None, None, x, None) == J.ERR_INVALID
    assert b"scratch" in lib.jacobi_last_error(None)
    # 3D dimensions just below 2^30: the partial count (~2^81) must not wrap
    # around int64 and slip past the scratch limit
    big = (1 << 30) - 1
    assert lib.jacobi_residual_noalloc(3, d3(big, big, big), x, None, None, x, None) == J.ERR_INVALID
    assert b"scratch" in lib.jacobi_last_error(None)
    assert lib.jacobi_residual_noalloc(3, d3(64, big, 8), x, None, None, x, None) == J.ERR_INVALID
    # the FP64 rate probe checks its arguments before any CUDA call
    v = ctypes.c_double()
    assert lib.jacobi_probe_fp64_rate(0, 3, 1, 16, ctypes.byref(v), None) == J.ERR_INVALID
    assert lib.jacobi_probe_fp64_rate(0, 8, 0, 16, ctypes.byref(v), None) == J.ERR_INVALID
    assert lib.jacobi_probe_fp64_rate(0, 8, 1, 0, ctypes.byref(v), None) == J.ERR_INVALID
    assert lib.jacobi_probe_fp64_rate(0, 8, 1, 16, None, None) == J.ERR_INVALID
    assert lib.jacobi_probe_fp64_rate(7, 8, 1, 16, ctypes.byref(v), None) == J.ERR_INVALID
