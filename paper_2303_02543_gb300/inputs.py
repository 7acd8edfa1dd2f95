"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds random-number generation and workload recipes only: no
Jacobi arithmetic.  Every array comes from a counter-based splitmix64 stream
keyed by (seed, array id), so the same bytes are handed to the CUDA library
and to the CPU oracle.

The paper runs its Jacobi proxy on a 1024x1024x768 domain split into cuboids
(section 4.3) and uses no public dataset; the recipes below are synthetic
stand-ins of the same shape family (2D and 3D grids, many blocks, uneven
batches, a Poisson arrival stream).

Array layout: interior-dense, numpy shape (nz, ny, nx) or (ny, nx), x fastest.
Boundary faces: a list of 2*ndim arrays ordered -x, +x, -y, +y, -z, +z; each
face lists its points with the remaining axes in order, lowest axis fastest
(2D: the x faces have ny values, the y faces nx values).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, array_id: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
        k = _mix(s + np.uint64(array_id & 0xFFFFFFFF) * _GAMMA + _GAMMA)
        return _mix(k ^ np.uint64(0xD1B54A32D192ED03))[0]


def u64_stream(seed: int, array_id: int, n: int, start: int = 0) -> np.ndarray:
    """Values start..start+n-1 of the splitmix64 stream for (seed, array_id)."""
    key = _key(seed, array_id)
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64) * _GAMMA + key
    return _mix(ctr)


def uniform(seed: int, array_id: int, n: int) -> np.ndarray:
    """n doubles uniform on [0, 1): top 53 bits of each draw times 2^-53."""
    return (u64_stream(seed, array_id, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, array_id: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller (cosine branch) on pairs of uniforms."""
    u = uniform(seed, array_id, 2 * n).reshape(n, 2)
    return np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


# Array ids within one problem.
ID_X0, ID_SOURCE, ID_FACE0 = 1, 2, 10   # faces use ID_FACE0 + face index


def face_shapes(dims):
    """Number of points of each Dirichlet face, ordered -x,+x,-y,+y,-z,+z."""
    nd = len(dims)
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    shapes = [ny * nz, ny * nz]
    if nd >= 2:
        shapes += [nx * nz, nx * nz]
    if nd == 3:
        shapes += [nx * ny, nx * ny]
    return shapes


@dataclass
class Problem:
    """One Jacobi problem: grid, decomposition and its input arrays."""
    dims: tuple            # (nx, ny[, nz]) interior points
    block: tuple           # block extent per axis (over-decomposition)
    faces: list            # Dirichlet values, one array per face
    source: np.ndarray | None
    x0: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.dims)

    @property
    def points(self):
        return int(np.prod(self.dims))

    @property
    def shape(self):
        return tuple(reversed(self.dims))


def make_problem(dims, block, seed, boundary="uniform", source="zero", x0="zero", const=0.0):
    """Build a problem: boundary in {"zero","uniform","const"}, source in
    {"zero","normal"}, x0 in {"zero","uniform"}."""
    dims = tuple(int(d) for d in dims)
    shape = tuple(reversed(dims))
    n = int(np.prod(dims))
    faces = []
    for i, m in enumerate(face_shapes(dims)):
        if boundary == "uniform":
            faces.append(uniform(seed, ID_FACE0 + i, m))
        elif boundary == "const":
            faces.append(np.full(m, float(const)))
        else:
            faces.append(np.zeros(m))
    f = normal(seed, ID_SOURCE, n).reshape(shape) if source == "normal" else None
    x = uniform(seed, ID_X0, n).reshape(shape) if x0 == "uniform" else None
    return Problem(dims, tuple(int(b) for b in block), faces, f, x,
                   {"seed": seed, "boundary": boundary, "source": source, "x0": x0})


# ---- workload recipes ------------------------------------------------------

def laplace_2d_small(seed=2304):
    """2D 5-point Laplace, 256x256 FP64, 4x4 blocks of 64x64, boundary and
    initial field uniform[0,1), no source; run 100 sweeps."""
    return make_problem((256, 256), (64, 64), seed, boundary="uniform", source="zero", x0="uniform")


def poisson_2d_large(seed=2305, n=8192, block=512):
    """2D 5-point Poisson, 8192x8192 FP64, 16x16 blocks of 512x512, boundary
    and initial field uniform[0,1), source normal(0,1); 1000 sweeps with a
    residual every 50."""
    return make_problem((n, n), (block, block), seed, boundary="uniform", source="normal", x0="uniform")


def poisson_3d(seed=2306, n=512, block=64):
    """3D 7-point Poisson, 512^3, blocks of 64^3, zero boundary, source
    normal(0,1), x0 = 0; solved to relative residual 1e-8."""
    return make_problem((n, n, n), (block, block, block), seed, boundary="zero", source="normal", x0="zero")


def log_uniform_sides(seed, array_id, count, lo, hi):
    """count integer sides with log(side) uniform on [log lo, log hi]."""
    u = uniform(seed, array_id, count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batched_2d(seed=2307, count=256, lo=64, hi=2048, block=128, size_scale=1.0):
    """count independent 2D Poisson problems; sides log-uniform on [lo, hi]
    drawn independently per axis (rectangular, uneven); blocks of block^2 with
    high-edge remainders; source normal(0,1), boundary uniform[0,1), x0 = 0.
    size_scale < 1 shrinks every side (for quick tests)."""
    sx = log_uniform_sides(seed, 100, count, lo, hi)
    sy = log_uniform_sides(seed, 101, count, lo, hi)
    probs = []
    for i in range(count):
        nx = max(1, int(round(sx[i] * size_scale)))
        ny = max(1, int(round(sy[i] * size_scale)))
        # a grid narrower than a block is a single block along that axis
        probs.append(make_problem((nx, ny), (min(block, nx), min(block, ny)), seed * 1000003 + i,
                                  boundary="uniform", source="normal", x0="zero"))
    return probs


@dataclass
class Arrival:
    t: float          # arrival time, seconds from stream start
    problem: Problem


def serving_stream(seed=2308, rate=10.0, window_s=60.0, lo2=128, hi2=4096, lo3=32, hi3=256,
                   block2=128, block3=32, max_requests=100000):
    """Poisson arrivals at `rate` req/s over `window_s` seconds; each request is
    a 2D square solve (side log-uniform [lo2, hi2]) or a 3D cube solve (side
    log-uniform [lo3, hi3]) with probability 1/2 each; source normal(0,1),
    boundary uniform[0,1), x0 = 0."""
    u_gap = uniform(seed, 200, max_requests)
    u_kind = uniform(seed, 201, max_requests)
    u_side = uniform(seed, 202, max_requests)
    out, t = [], 0.0
    for i in range(max_requests):
        t += -math.log1p(-u_gap[i]) / rate
        if t > window_s:
            break
        if u_kind[i] < 0.5:
            side = int(round(math.exp(math.log(lo2) + u_side[i] * (math.log(hi2) - math.log(lo2)))))
            b = min(block2, side)
            dims, block = (side, side), (b, b)
        else:
            side = int(round(math.exp(math.log(lo3) + u_side[i] * (math.log(hi3) - math.log(lo3)))))
            b = min(block3, side)
            dims, block = (side, side, side), (b, b, b)
        p = make_problem(dims, block, seed * 1000003 + i, boundary="uniform", source="normal", x0="zero")
        p.meta["arrival"] = t
        out.append(Arrival(t, p))
    return out
