"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (and the seeded input generators).  Run from the repo root:

    python tests/golden/make_golden.py

Fixture laplace_2d_256_100.json: the 2D 5-point Laplace workload (256x256
interior, boundary and initial field uniform[0,1) from seed 2304, no source)
after 100 Jacobi sweeps -- the fixed-iteration Jacobi proxy of section 4.3 on
a 2D grid.  It stores exact (hex) values at sampled points plus the sums of
squares of the residual and of b.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2303_02543_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def sample_points(shape, count, seed):
    ny, nx = shape
    u = inputs.u64_stream(seed, 300, 2 * count)
    ys = (u[:count] % np.uint64(ny)).astype(int)
    xs = (u[count:] % np.uint64(nx)).astype(int)
    fixed = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (63, 64), (64, 63), (127, 128)]
    return fixed + list(zip(ys.tolist(), xs.tolist()))


def main():
    p = inputs.laplace_2d_small()
    x = oracle.sweeps(p.dims, p.faces, p.source, p.x0, 100)
    rss, bss = oracle.residual(p.dims, p.faces, p.source, x)
    pts = sample_points(p.shape, 250, 7)
    doc = {
        "citation": "section 4.3: fixed number of Jacobi iterations on a decomposed domain "
                    "(2D 5-point reading); workload 256x256 Laplace, 100 sweeps",
        "workload": "laplace_2d_small(seed=2304): 256x256, blocks 64x64, g~U[0,1), x0~U[0,1), f=0",
        "sweeps": 100,
        "points": [[y, xx, float(x[y, xx]).hex()] for y, xx in pts],
        "rss": float(rss).hex(),
        "bss": float(bss).hex(),
    }
    pts_txt = ",\n".join("  " + json.dumps(q) for q in doc.pop("points"))
    body = json.dumps(doc, indent=1)[:-2]
    with open(os.path.join(HERE, "laplace_2d_256_100.json"), "w") as fh:
        fh.write(body + ',\n "points": [\n' + pts_txt + "\n ]\n}\n")


if __name__ == "__main__":
    main()
