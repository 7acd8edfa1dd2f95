"""Thin Python binding of the C ABI in include/jacobi.h (argument marshalling
only: every step of the Jacobi path runs in the CUDA library).

The functions named ``jacobi_*`` mirror the C entry points one to one; the
``Solver`` class wraps them for convenience.  PyTorch supplies the device
memory (the library's allocations are routed to torch's caching allocator)
and the stream (torch's current stream).  There is no CPU fallback: if the
CUDA library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

from . import build as _build

F64, F32_REFINE, BF16_REFINE, BF16_REFINE_R16 = 0, 1, 2, 3
DTYPES = {"f64": F64, "f32_refine": F32_REFINE, "bf16_refine": BF16_REFINE, "bf16r16_refine": BF16_REFINE_R16}
BC_ZERO, BC_CONST, BC_FACES = 0, 1, 2

STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NOT_CONVERGED",
          5: "ERR_DIVERGED", 6: "ERR_TIMEOUT", 7: "ERR_BUSY"}
OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_TIMEOUT, ERR_BUSY = range(8)

# Every symbol declared in include/jacobi.h.
EXPORTS = ["jacobi_set_allocator", "jacobi_create", "jacobi_sweep", "jacobi_residual", "jacobi_solve",
           "jacobi_get_field", "jacobi_set_field", "jacobi_set_source", "jacobi_set_option",
           "jacobi_get_option", "jacobi_profile", "jacobi_device_bytes", "jacobi_destroy",
           "jacobi_last_error", "jacobi_version", "jacobi_residual_noalloc", "jacobi_probe_fp64_rate",
           "jacobi_batch_create", "jacobi_batch_solve", "jacobi_batch_get_field",
           "jacobi_server_create", "jacobi_server_set_option", "jacobi_server_submit", "jacobi_server_poll",
           "jacobi_server_wait", "jacobi_server_get_stats", "jacobi_server_destroy"]


class JacobiError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Boundary(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("value", ctypes.c_double), ("faces", ctypes.c_void_p * 6)]


class Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("block", ctypes.c_int64 * 3),
                ("bc", Boundary), ("source", ctypes.c_void_p), ("x0", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "rejected", "active", "queued",
                                               "bytes_in_use", "budget_bytes", "steps")] + [("lups", ctypes.c_double)]
                + [("evictions", ctypes.c_int64), ("resumed", ctypes.c_int64)])


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("sweeps", ctypes.c_int64),
                ("rel", ctypes.c_double), ("seconds", ctypes.c_double)]


_lib = None
_alloc_cb = None
_free_cb = None
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with "
                           "`python -m paper_2303_02543_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    vp, i64, i64p, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    sig = {
        "jacobi_set_allocator": (None, [ALLOC_FN, FREE_FN, vp]),
        "jacobi_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64p, i64p, ctypes.c_int,
                                          ctypes.POINTER(Boundary), vp, vp, vp]),
        "jacobi_sweep": (ctypes.c_int, [vp, i64]),
        "jacobi_residual": (ctypes.c_int, [vp, dp, dp]),
        "jacobi_solve": (ctypes.c_int, [vp, ctypes.c_double, i64, i64p, dp]),
        "jacobi_get_field": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "jacobi_set_field": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "jacobi_set_source": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "jacobi_set_option": (ctypes.c_int, [vp, ctypes.c_char_p, i64]),
        "jacobi_get_option": (ctypes.c_int, [vp, ctypes.c_char_p, i64p]),
        "jacobi_profile": (ctypes.c_int, [vp, ctypes.c_char_p, dp, i64p, ctypes.c_int]),
        "jacobi_device_bytes": (ctypes.c_int, [vp, i64p]),
        "jacobi_destroy": (None, [vp]),
        "jacobi_last_error": (ctypes.c_char_p, [vp]),
        "jacobi_version": (ctypes.c_int, []),
        "jacobi_residual_noalloc": (ctypes.c_int, [ctypes.c_int, i64p, vp, vp, ctypes.POINTER(vp), vp, vp]),
        "jacobi_probe_fp64_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, dp, vp]),
        "jacobi_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(Problem),
                                                ctypes.c_int, vp]),
        "jacobi_batch_solve": (ctypes.c_int, [vp, ctypes.c_double, i64, ctypes.POINTER(Result)]),
        "jacobi_batch_get_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
        "jacobi_server_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64, ctypes.c_int, vp]),
        "jacobi_server_set_option": (ctypes.c_int, [vp, ctypes.c_char_p, i64]),
        "jacobi_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(Problem), ctypes.c_double, i64,
                                                 ctypes.POINTER(ctypes.c_uint64)]),
        "jacobi_server_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(Result), vp]),
        "jacobi_server_wait": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double]),
        "jacobi_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
        "jacobi_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator.

    The ctypes trampolines are created once and kept for the life of the
    process: a context keeps the hooks it was created with, so replacing them
    while a context is alive would leave it calling freed code."""
    global _alloc_cb, _free_cb
    lib = load()
    if not enable:
        lib.jacobi_set_allocator(ALLOC_FN(), FREE_FN(), None)
        return
    if _alloc_cb is not None:
        lib.jacobi_set_allocator(_alloc_cb, _free_cb, None)
        return
    import torch

    def _alloc(nbytes, stream, _user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                                          stream=int(stream or 0)))
        except Exception:  # noqa: BLE001 - reported to C as a NULL allocation (JACOBI_ERR_OOM)
            return None

    def _free(ptr, _stream, _user):
        if ptr and not sys.is_finalizing():
            torch.cuda.caching_allocator_delete(int(ptr))

    _alloc_cb, _free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
    lib.jacobi_set_allocator(_alloc_cb, _free_cb, None)


def _check(status, handle=None):
    if status != OK:
        msg = load().jacobi_last_error(handle)
        raise JacobiError(status, msg.decode() if msg else "")
    return status


def _ptr(a, shape, writable=False):
    """Host numpy array or torch tensor holding one interior-dense field of
    `shape` -> (pointer, on_device).  The C side trusts the size, so a
    mismatch in size, dtype, contiguity or device is refused here."""
    n = int(np.prod(shape))
    if hasattr(a, "data_ptr"):  # torch tensor: device or (pinned) host memory
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"field tensor must be contiguous float64 with {n} elements "
                             f"(got {a.dtype}, {tuple(a.shape)}, contiguous={a.is_contiguous()})")
        if a.is_cuda and a.device.index != torch.cuda.current_device():
            raise ValueError(f"field tensor is on {a.device}, the library runs on cuda:{torch.cuda.current_device()}")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
        raise ValueError(f"field array must be a C-contiguous float64 numpy array with {n} elements")
    if writable and not a.flags.writeable:
        raise ValueError("output field array is read-only")
    return ctypes.c_void_p(a.ctypes.data), 0


def default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


# ---- C entry points, one to one -------------------------------------------

def jacobi_version():
    return load().jacobi_version()


def jacobi_create(ndim, dims, block, dtype, bc=None, source=None, x0=None, stream=None):
    lib = load()
    dl, bl = list(dims)[:3], list(block)[:3]  # the C side validates ndim against 2..3
    d = (ctypes.c_int64 * 3)(*(dl + [1] * (3 - len(dl))))
    b = (ctypes.c_int64 * 3)(*(bl + [1] * (3 - len(bl))))
    h = ctypes.c_void_p()
    st = lib.jacobi_create(ctypes.byref(h), ndim, d, b, dtype, None if bc is None else ctypes.byref(bc),
                           source, x0, stream)
    _check(st, None)
    return h


def jacobi_sweep(h, n):
    return _check(load().jacobi_sweep(h, int(n)), h)


def jacobi_residual(h):
    rel, ab = ctypes.c_double(), ctypes.c_double()
    _check(load().jacobi_residual(h, ctypes.byref(rel), ctypes.byref(ab)), h)
    return rel.value, ab.value


def jacobi_solve(h, tol, max_sweeps):
    sw, rel = ctypes.c_int64(), ctypes.c_double()
    st = load().jacobi_solve(h, float(tol), int(max_sweeps), ctypes.byref(sw), ctypes.byref(rel))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
        _check(st, h)
    return st, sw.value, rel.value


def jacobi_get_field(h, out_ptr, on_device):
    return _check(load().jacobi_get_field(h, out_ptr, int(on_device)), h)


def jacobi_set_field(h, in_ptr, on_device):
    return _check(load().jacobi_set_field(h, in_ptr, int(on_device)), h)


def jacobi_set_source(h, in_ptr, on_device):
    return _check(load().jacobi_set_source(h, in_ptr, int(on_device)), h)


def jacobi_set_option(h, key, value):
    return _check(load().jacobi_set_option(h, key.encode(), int(value)), h)


def jacobi_get_option(h, key):
    v = ctypes.c_int64()
    _check(load().jacobi_get_option(h, key.encode(), ctypes.byref(v)), h)
    return v.value


def jacobi_profile(h, kernel, reset=False):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load().jacobi_profile(h, kernel.encode(), ctypes.byref(ms), ctypes.byref(n), int(bool(reset))), h)
    return ms.value, n.value


def jacobi_device_bytes(h):
    v = ctypes.c_int64()
    _check(load().jacobi_device_bytes(h, ctypes.byref(v)), h)
    return v.value


def jacobi_destroy(h):
    if h:
        load().jacobi_destroy(h)


def jacobi_residual_noalloc(ndim, dims, x_ptr, f_ptr, face_ptrs, rss_ptr, stream=None):
    """Residual sum of squares of an interior-dense device field into the
    device double at rss_ptr, using only the library's fixed scratch."""
    dl = list(dims)[:3]
    d = (ctypes.c_int64 * 3)(*(dl + [1] * (3 - len(dl))))
    fp = None
    if face_ptrs is not None:
        fp = (ctypes.c_void_p * 6)(*(list(face_ptrs) + [None] * (6 - len(face_ptrs))))
    return _check(load().jacobi_residual_noalloc(int(ndim), d, x_ptr, f_ptr, fp, rss_ptr, stream), None)


def jacobi_probe_fp64_rate(form=0, chains=8, ctas_per_sm=8, iters=4096, stream=None):
    """FP64 lane operations per second on the current device of one
    instruction form (0: fma.rn.f64 with immediate multiplier 1.0; 1: with a
    register multiplier 1.0; 2: add.rn.f64; 3: mul.rn.f64; 4: fma.rn.f64 with
    the multiplier 1.0 in constant memory)."""
    v = ctypes.c_double()
    _check(load().jacobi_probe_fp64_rate(int(form), int(chains), int(ctas_per_sm), int(iters), ctypes.byref(v),
                                         stream), None)
    return v.value


def jacobi_batch_create(problems, dtype, stream=None):
    """problems: a ctypes array of Problem."""
    h = ctypes.c_void_p()
    _check(load().jacobi_batch_create(ctypes.byref(h), len(problems), problems, int(dtype), stream), None)
    return h


def jacobi_batch_solve(h, tol, max_sweeps, n):
    res = (Result * n)()
    st = load().jacobi_batch_solve(h, float(tol), int(max_sweeps), res)
    if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
        _check(st, h)
    return st, res


def jacobi_batch_get_field(h, i, out_ptr, on_device):
    return _check(load().jacobi_batch_get_field(h, int(i), out_ptr, int(on_device)), h)


def jacobi_last_error(h=None):
    m = load().jacobi_last_error(h)
    return m.decode() if m else ""


# ---- convenience wrapper -------------------------------------------------

def face_sizes(dims):
    """Values per Dirichlet face, in the header's face order (x-, x+, y-, y+,
    z-, z+), for a grid of dims (nx, ny[, nz])."""
    n = list(dims) + [1] * (3 - len(dims))
    return [n[1] * n[2], n[1] * n[2], n[0] * n[2], n[0] * n[2], n[0] * n[1], n[0] * n[1]][:2 * len(dims)]


def _host_input(v, n, what):
    """Contiguous float64 copy (or view) of a host input that must hold n
    values: the C side reads exactly n, so any other size is refused."""
    a = np.ascontiguousarray(v, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"{what} has {a.size} values; the grid needs {n}")
    return a


def make_boundary(faces=None, value=None, dims=None):
    """Boundary struct from a list of face arrays (host) or a constant.  With
    dims, every face's size is checked against the grid."""
    bc = Boundary()
    keep = []
    if faces is not None:
        bc.kind = BC_FACES
        sizes = face_sizes(dims) if dims is not None else [None] * 6
        if len(faces) > len(sizes):
            raise ValueError(f"{len(faces)} faces given; the grid has {len(sizes)}")
        for i, f in enumerate(faces):
            if f is None:
                bc.faces[i] = None
                continue
            arr = (np.ascontiguousarray(f, dtype=np.float64) if sizes[i] is None
                   else _host_input(f, sizes[i], f"face {i}"))
            keep.append(arr)
            bc.faces[i] = arr.ctypes.data
    elif value is not None:
        bc.kind, bc.value = BC_CONST, float(value)
    else:
        bc.kind = BC_ZERO
    return bc, keep


class Solver:
    """One grid: Solver(dims, block, dtype="f64", faces=..., source=..., x0=...)."""

    def __init__(self, dims, block, dtype="f64", faces=None, bc_value=None, source=None, x0=None,
                 stream=None, torch_alloc=True, **options):
        self.dims = tuple(int(d) for d in dims)
        self.ndim = len(self.dims)
        self.shape = tuple(reversed(self.dims))
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        if torch_alloc:
            use_torch_allocator(True)
        bc, keep = make_boundary(faces, bc_value, self.dims)
        npts = int(np.prod(self.dims))
        src = None if source is None else _host_input(source, npts, "source")
        xx = None if x0 is None else _host_input(x0, npts, "x0")
        self.stream = default_stream() if stream is None else stream
        self.h = jacobi_create(self.ndim, self.dims, block, self.dtype, bc,
                               None if src is None else src.ctypes.data,
                               None if xx is None else xx.ctypes.data, self.stream)
        del keep
        for k, v in options.items():
            self.set_option(k, v)

    def sweep(self, n):
        jacobi_sweep(self.h, n)

    def residual(self):
        return jacobi_residual(self.h)

    def solve(self, tol, max_sweeps):
        return jacobi_solve(self.h, tol, max_sweeps)

    def field(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        p, dev = _ptr(out, self.shape, writable=True)
        jacobi_get_field(self.h, p, dev)
        return out

    def set_field(self, x):
        if not hasattr(x, "data_ptr"):
            x = np.ascontiguousarray(x, dtype=np.float64)
        p, dev = _ptr(x, self.shape)
        jacobi_set_field(self.h, p, dev)

    def set_source(self, f):
        if not hasattr(f, "data_ptr"):
            f = np.ascontiguousarray(f, dtype=np.float64)
        p, dev = _ptr(f, self.shape)
        jacobi_set_source(self.h, p, dev)

    def set_option(self, key, value):
        jacobi_set_option(self.h, key, value)

    def get_option(self, key):
        return jacobi_get_option(self.h, key)

    def profile(self, kernel, reset=False):
        return jacobi_profile(self.h, kernel, reset)

    def device_bytes(self):
        return jacobi_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            jacobi_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        if not sys.is_finalizing():
            try:
                self.close()
            except Exception:  # noqa: BLE001
                pass


class Batch:
    """Many independent grids in one context: Batch(problems, dtype=...) where
    each problem has .dims, .block, .faces, .source, .x0 (host numpy)."""

    def __init__(self, problems, dtype="f32_refine", stream=None, torch_alloc=True, **options):
        self.n = len(problems)
        self.shapes = [tuple(reversed(tuple(p.dims))) for p in problems]
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        if torch_alloc:
            use_torch_allocator(True)
        arr = (Problem * self.n)()
        keep = []
        for i, p in enumerate(problems):
            arr[i] = _problem_struct(p, keep)
        self.stream = default_stream() if stream is None else stream
        self.h = jacobi_batch_create(arr, self.dtype, self.stream)
        del keep
        for k, v in options.items():
            jacobi_set_option(self.h, k, v)

    def solve(self, tol, max_sweeps):
        st, res = jacobi_batch_solve(self.h, tol, max_sweeps, self.n)
        return st, [(r.status, r.sweeps, r.rel, r.seconds) for r in res]

    def sweep(self, n):
        jacobi_sweep(self.h, n)

    def field(self, i, out=None):
        if out is None:
            out = np.empty(self.shapes[i], dtype=np.float64)
        p, dev = _ptr(out, self.shapes[i], writable=True)
        jacobi_batch_get_field(self.h, i, p, dev)
        return out

    def set_option(self, key, value):
        jacobi_set_option(self.h, key, value)

    def profile(self, kernel, reset=False):
        return jacobi_profile(self.h, kernel, reset)

    def close(self):
        if getattr(self, "h", None):
            jacobi_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        if not sys.is_finalizing():
            try:
                self.close()
            except Exception:  # noqa: BLE001
                pass


def _problem_struct(p, keep):
    """Problem struct for an inputs.Problem-like object (host numpy arrays)."""
    ps = Problem()
    dims, blk = list(p.dims), list(p.block)
    ps.ndim = len(dims)
    for a in range(3):
        ps.dims[a] = dims[a] if a < len(dims) else 1
        ps.block[a] = blk[a] if a < len(blk) else 1
    bc, k = make_boundary(p.faces, dims=dims)
    keep.append(k)
    ps.bc = bc
    npts = int(np.prod(dims))
    for name in ("source", "x0"):
        v = getattr(p, name)
        if v is None:
            setattr(ps, name, None)
        else:
            a_ = _host_input(v, npts, name)
            keep.append(a_)
            setattr(ps, name, a_.ctypes.data)
    return ps


class Server:
    """Continuous-batching server: Server(dtype, budget_bytes, max_slots)."""

    def __init__(self, dtype="f32_refine", budget_bytes=1 << 30, max_slots=64, stream=None, torch_alloc=True,
                 **options):
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        if torch_alloc:
            use_torch_allocator(True)
        self.stream = default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        _check(load().jacobi_server_create(ctypes.byref(h), self.dtype, int(budget_bytes), int(max_slots),
                                           self.stream), None)
        self.h = h
        self.shapes = {}
        for k, v in options.items():
            _check(load().jacobi_server_set_option(self.h, k.encode(), int(v)), None)

    def submit(self, problem, tol, max_sweeps):
        keep = []
        ps = _problem_struct(problem, keep)
        t = ctypes.c_uint64()
        _check(load().jacobi_server_submit(self.h, ctypes.byref(ps), float(tol), int(max_sweeps), ctypes.byref(t)),
               None)
        self.shapes[t.value] = tuple(reversed(tuple(problem.dims)))
        return t.value

    def poll(self, ticket, want_field=True):
        """None while pending, else (status, sweeps, rel, seconds, field)."""
        r = Result()
        out = np.empty(self.shapes[ticket], dtype=np.float64) if want_field else None
        st = load().jacobi_server_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r),
                                       None if out is None else out.ctypes.data)
        if st == ERR_BUSY:
            return None
        _check(st, None)
        del self.shapes[ticket]
        return r.status, r.sweeps, r.rel, r.seconds, out

    def wait(self, ticket, timeout_s=60.0):
        return load().jacobi_server_wait(self.h, ctypes.c_uint64(ticket), float(timeout_s)) == OK

    def stats(self):
        st = ServerStats()
        _check(load().jacobi_server_get_stats(self.h, ctypes.byref(st)), None)
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().jacobi_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        if not sys.is_finalizing():
            try:
                self.close()
            except Exception:  # noqa: BLE001
                pass
