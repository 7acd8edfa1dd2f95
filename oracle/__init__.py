"""Jacobi oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU Jacobi relaxation (section 4.3's Jacobi proxy: fixed sweeps of
the Jacobi method on a decomposed 3D domain; the decomposition of section 4.4
does not change the iterate, so the oracle works on one monolithic grid).  The
arithmetic lives in ``jacobi_oracle.c``; this module only compiles it and
marshals numpy arrays.  ``dense.py`` holds a second, independent check built on
dense matrices.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline
leg may import this package.  It never imports the CUDA package and the CUDA
package never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libjacobi_oracle.so")
_lib = None

OK, INVALID, OOM, NOT_CONVERGED, DIVERGED = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, OpenMP, no FMA contraction."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = _load_path(build())
    return _lib


def _load_path(path):
    lib = ctypes.CDLL(path)
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.c_void_p
    lib.jo_sweeps.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.c_int64, ctypes.c_int]
    lib.jo_residual.argtypes = [ctypes.c_int, i64p, dp, dp, dp, dp, dp, dp, ctypes.c_int]
    lib.jo_solve.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.c_double, ctypes.c_int64,
                             ctypes.c_int64, dp, dp, ctypes.c_int]
    lib.jo_refine_solve.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_double, ctypes.c_int64, dp, dp,
                                    ctypes.c_int]
    lib.jo_round_bf16.argtypes = [ctypes.c_float]
    lib.jo_round_bf16.restype = ctypes.c_float
    lib.jo_max_threads.restype = ctypes.c_int
    return lib


class use_library:
    """Context manager that points this module at another build of the oracle
    source (the pin-strength tests compile deliberately broken copies)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = None
        lib = _load_path(self.path)
        _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_source(src_text: str, out_path: str) -> str:
    """Compile C source text with the oracle's flags into out_path."""
    c_path = out_path + ".c"
    with open(c_path, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                    "-shared", "-fPIC", "-o", out_path, c_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def max_threads() -> int:
    return int(_load().jo_max_threads())


class _Args:
    """Holds contiguous float64 copies and the ctypes pointers into them."""

    def __init__(self, dims, faces, f):
        self.ndim = len(dims)
        self.dims = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
        self.keep = []
        ptrs = (ctypes.c_void_p * 6)()
        for i in range(6):
            face = None if faces is None or i >= len(faces) else faces[i]
            if face is None:
                ptrs[i] = None
            else:
                arr = np.ascontiguousarray(face, dtype=np.float64)
                self.keep.append(arr)
                ptrs[i] = arr.ctypes.data
        self.faces = ptrs
        self.f = None
        if f is not None:
            farr = np.ascontiguousarray(f, dtype=np.float64)
            self.keep.append(farr)
            self.f = farr.ctypes.data


def _field(x, dims):
    shape = tuple(reversed(tuple(dims)))
    if x is None:
        return np.zeros(shape, dtype=np.float64)
    return np.array(x, dtype=np.float64, copy=True, order="C").reshape(shape)


def sweeps(dims, faces, f, x0, nsweeps, threads=0):
    """Return x after ``nsweeps`` Jacobi sweeps from x0 (dims = (nx[, ny[, nz]]);
    arrays are interior-dense, shape reversed(dims), x fastest)."""
    a = _Args(dims, faces, f)
    x = _field(x0, dims)
    st = _load().jo_sweeps(a.ndim, a.dims, a.faces, a.f, x.ctypes.data, int(nsweeps), int(threads))
    if st != OK:
        raise RuntimeError(f"oracle sweeps failed: {st}")
    return x


def residual(dims, faces, f, x, threads=0, want_r=False):
    """(rss, bss[, r]): sum of squares of r = b - A x and of b."""
    a = _Args(dims, faces, f)
    xa = _field(x, dims)
    rss, bss = ctypes.c_double(), ctypes.c_double()
    r = np.empty_like(xa) if want_r else None
    st = _load().jo_residual(a.ndim, a.dims, a.faces, a.f, xa.ctypes.data, ctypes.addressof(rss),
                             ctypes.addressof(bss), None if r is None else r.ctypes.data, int(threads))
    if st != OK:
        raise RuntimeError(f"oracle residual failed: {st}")
    return (rss.value, bss.value, r) if want_r else (rss.value, bss.value)


def relative_residual(dims, faces, f, x, threads=0):
    rss, bss = residual(dims, faces, f, x, threads)
    return float(np.sqrt(rss) / np.sqrt(bss)) if bss > 0 else float(np.sqrt(rss))


def solve(dims, faces, f, x0, tol, max_sweeps, check_every, threads=0):
    """Plain FP64 Jacobi to rel <= tol, checked every ``check_every`` sweeps.
    Returns (status, x, sweeps, rel)."""
    a = _Args(dims, faces, f)
    x = _field(x0, dims)
    sw, rel = ctypes.c_int64(), ctypes.c_double()
    st = _load().jo_solve(a.ndim, a.dims, a.faces, a.f, x.ctypes.data, float(tol), int(max_sweeps),
                          int(check_every), ctypes.addressof(sw), ctypes.addressof(rel), int(threads))
    if st == INVALID:
        raise ValueError("oracle solve: invalid arguments")
    return st, x, sw.value, rel.value


def refine_solve(dims, faces, f, x0, tol, max_sweeps, period, e_bf16=False, r_bf16=False, threads=0):
    """FP64 iterative refinement with float (or bfloat16-stored) inner sweeps.
    Returns (status, x, inner_sweeps, rel)."""
    a = _Args(dims, faces, f)
    x = _field(x0, dims)
    sw, rel = ctypes.c_int64(), ctypes.c_double()
    st = _load().jo_refine_solve(a.ndim, a.dims, a.faces, a.f, x.ctypes.data, int(bool(e_bf16)),
                                 int(bool(r_bf16)), int(period), float(tol), int(max_sweeps),
                                 ctypes.addressof(sw), ctypes.addressof(rel), int(threads))
    if st == INVALID:
        raise ValueError("oracle refine_solve: invalid arguments")
    return st, x, sw.value, rel.value


def round_bf16(v: float) -> float:
    return float(_load().jo_round_bf16(ctypes.c_float(v)))
