"""Dense-matrix Jacobi checker -- TEST INFRASTRUCTURE ONLY.

An implementation of the same method written a second, independent way: the
grid operator is assembled as an explicit dense matrix A (negative Laplacian,
unit spacing, Dirichlet) with right-hand side b = f + (Dirichlet values of
ghost neighbours), and Jacobi is iterated in matrix form,
x <- x + D^-1 (b - A x) with D = diag(A) = 2d I.  Only usable on tiny grids.
"""
from __future__ import annotations

import itertools

import numpy as np


def _index(dims):
    """Map interior coordinates (x fastest) to a row of A."""
    return {c: i for i, c in enumerate(itertools.product(*[range(n) for n in reversed(dims)]))}


def assemble(dims, faces, f):
    """Return (A, b) for the grid dims=(nx[, ny[, nz]]).  Coordinates are
    handled as (.., y, x) tuples to match the interior-dense layout."""
    nd = len(dims)
    n = int(np.prod(dims))
    A = np.zeros((n, n))
    b = np.zeros(n) if f is None else np.array(f, dtype=np.float64).reshape(-1).copy()
    idx = _index(dims)
    rdims = list(reversed(dims))           # (.., ny, nx)
    for coord, row in idx.items():
        A[row, row] = 2.0 * nd
        for axis in range(nd):             # axis 0 = x
            ax = nd - 1 - axis             # position of that axis in coord
            for sgn in (-1, +1):
                nb = list(coord)
                nb[ax] += sgn
                if 0 <= nb[ax] < rdims[ax]:
                    A[row, idx[tuple(nb)]] -= 1.0
                else:
                    b[row] += _face_value(dims, faces, axis, sgn, coord)
    return A, b


def _face_value(dims, faces, axis, sgn, coord):
    """Dirichlet value on face (axis, sgn) next to interior point coord."""
    if faces is None:
        return 0.0
    face = faces[2 * axis + (0 if sgn < 0 else 1)]
    if face is None:
        return 0.0
    nd = len(dims)
    pos = list(reversed(coord))            # (x, y, z)
    rest = [pos[a] for a in range(nd) if a != axis]
    rest_n = [dims[a] for a in range(nd) if a != axis]
    k, mult = 0, 1
    for c, m in zip(rest, rest_n):
        k += c * mult
        mult *= m
    return float(np.asarray(face).reshape(-1)[k])


def jacobi_matrix_form(A, b, x0, k):
    """k Jacobi iterations written as x <- x + D^-1 (b - A x)."""
    d = np.diag(A)
    x = np.array(x0, dtype=np.float64).reshape(-1).copy()
    for _ in range(k):
        x = x + (b - A @ x) / d
    return x


def iteration_spectral_radius(A):
    """rho(I - D^-1 A) from a dense eigenvalue solve."""
    M = np.eye(A.shape[0]) - A / np.diag(A)[:, None]
    return float(np.max(np.abs(np.linalg.eigvals(M))))
