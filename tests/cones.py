"""Oracle values of single points of a large run, from their dependency cones.

After k Jacobi sweeps the value at a point depends only on the initial field,
the source and the Dirichlet values within distance k of it (one grid step per
sweep along every axis).  A refinement step of k inner sweeps followed by the
outer update reaches k + 1 further.  So the oracle, run on a window of radius
R around the point, returns that point's value of the full-size run exactly,
provided R covers the cone.  Where the window meets the domain boundary it
uses the real Dirichlet values; on its other sides it uses the initial field
just outside it.  Those values are wrong after the first sweep, but their
error travels inward one step per sweep and never reaches the centre.  The
test compares the GPU's value at the point with the oracle's, bit for bit.

This is test infrastructure: it calls only `oracle` and numpy.
"""
import numpy as np


def window(p, center, radius):
    """Problem restricted to the box of the given radius around `center`
    (x, y[, z]), clipped to the domain.  Returns (dims, faces, source, x0,
    index), where index is the centre's position (x, y[, z]) in the window."""
    nd = p.ndim
    dims = p.dims
    lo = [max(0, center[a] - radius) for a in range(nd)]
    hi = [min(dims[a] - 1, center[a] + radius) for a in range(nd)]
    wd = tuple(hi[a] - lo[a] + 1 for a in range(nd))
    x0 = p.x0 if p.x0 is not None else np.zeros(p.shape)
    if nd == 2:
        sl = (slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
    else:
        sl = (slice(lo[2], hi[2] + 1), slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
    src = None if p.source is None else np.ascontiguousarray(p.source[sl])
    xw = np.ascontiguousarray(x0[sl])
    faces = []
    if nd == 2:
        nx, ny = dims
        ys, xs = np.arange(lo[1], hi[1] + 1), np.arange(lo[0], hi[0] + 1)
        faces.append(p.faces[0][ys] if lo[0] == 0 else x0[ys, lo[0] - 1])
        faces.append(p.faces[1][ys] if hi[0] == nx - 1 else x0[ys, hi[0] + 1])
        faces.append(p.faces[2][xs] if lo[1] == 0 else x0[lo[1] - 1, xs])
        faces.append(p.faces[3][xs] if hi[1] == ny - 1 else x0[hi[1] + 1, xs])
    else:
        nx, ny, nz = dims
        xs, ys, zs = (np.arange(lo[a], hi[a] + 1) for a in range(3))
        fx = lambda q: p.faces[q].reshape(nz, ny)  # x faces: y fastest, then z
        fy = lambda q: p.faces[q].reshape(nz, nx)  # y faces: x fastest, then z
        fz = lambda q: p.faces[q].reshape(ny, nx)  # z faces: x fastest, then y
        zz, yy = np.meshgrid(zs, ys, indexing="ij")
        faces.append((fx(0)[zz, yy] if lo[0] == 0 else x0[zz, yy, lo[0] - 1]).ravel())
        faces.append((fx(1)[zz, yy] if hi[0] == nx - 1 else x0[zz, yy, hi[0] + 1]).ravel())
        zz, xx = np.meshgrid(zs, xs, indexing="ij")
        faces.append((fy(2)[zz, xx] if lo[1] == 0 else x0[zz, lo[1] - 1, xx]).ravel())
        faces.append((fy(3)[zz, xx] if hi[1] == ny - 1 else x0[zz, hi[1] + 1, xx]).ravel())
        yy, xx = np.meshgrid(ys, xs, indexing="ij")
        faces.append((fz(4)[yy, xx] if lo[2] == 0 else x0[lo[2] - 1, yy, xx]).ravel())
        faces.append((fz(5)[yy, xx] if hi[2] == nz - 1 else x0[hi[2] + 1, yy, xx]).ravel())
    faces = [np.ascontiguousarray(f, dtype=np.float64) for f in faces]
    index = tuple(center[a] - lo[a] for a in range(nd))
    return wd, faces, src, xw, index


def value_at(field, index):
    """field[z, y, x] (or [y, x]) at index (x, y[, z])."""
    return field[tuple(reversed(index))]


def sample_points(dims, blocks, count, seed):
    """Corners, points on both sides of block seams and domain edges, and
    seeded interior points."""
    nd = len(dims)
    rng = np.random.default_rng(seed)
    pts = set()
    for corner in range(1 << nd):
        pts.add(tuple((dims[a] - 1) if (corner >> a) & 1 else 0 for a in range(nd)))
    for a in range(nd):
        if dims[a] > blocks[a]:
            seam = blocks[a]
            for d in (seam - 1, seam):
                c = [dims[b] // 2 for b in range(nd)]
                c[a] = d
                pts.add(tuple(c))
    while len(pts) < count:
        pts.add(tuple(int(rng.integers(0, dims[a])) for a in range(nd)))
    return sorted(pts)
