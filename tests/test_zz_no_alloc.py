"""The allocation-free residual entry point, through the C ABI.

jacobi_residual_noalloc serves callers that cannot call cudaMalloc (device
memory owned in full by another runtime, or loops that must never stall the
device on an allocation).  Its scratch is a fixed device array inside the
library.  This file is named so that pytest collects it last; it must pass
alone in a fresh process and after every other test.
"""
import math

import numpy as np
import pytest

from paper_2303_02543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_02543_gb300 import build  # noqa: E402
from paper_2303_02543_gb300 import jacobi as J  # noqa: E402

build.build()


def device_inputs(p, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    fd = None if p.source is None else torch.from_numpy(np.ascontiguousarray(p.source)).cuda()
    faces = [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in p.faces]
    return xd, fd, faces


def noalloc_rss(p, xd, fd, faces):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    J.jacobi_residual_noalloc(p.ndim, p.dims, xd.data_ptr(), None if fd is None else fd.data_ptr(),
                              [g.data_ptr() for g in faces], out.data_ptr(), stream)
    torch.cuda.synchronize()
    return float(out.item())


@pytest.mark.parametrize("dims,block", [((300, 190), (64, 64)), ((300, 190), (300, 190)),
                                        ((70, 40, 30), (64, 16, 8)), ((129, 1), (129, 1))])
def test_noalloc_matches_context_residual_twice(dims, block):
    p = inputs.make_problem(dims, block, 61, boundary="uniform", source="normal", x0="uniform")
    with J.Solver(p.dims, p.block, faces=p.faces, source=p.source, x0=p.x0) as s:
        for sweeps in (3, 5):  # two calls in a row on different fields
            s.sweep(sweeps)
            _, ab = s.residual()
            ref = ab * ab
            xd, fd, faces = device_inputs(p, s.field())
            got = noalloc_rss(p, xd, fd, faces)
            assert abs(got - ref) <= 1e-12 * ref
            # same partial layout and reduction tree: the sums agree bit for
            # bit (jacobi_residual reports the correctly rounded sqrt)
            assert math.sqrt(got) == ab


def test_noalloc_zero_source_and_faces():
    p = inputs.make_problem((100, 80), (100, 80), 62, boundary="zero", source="zero", x0="uniform")
    with J.Solver(p.dims, p.block, x0=p.x0) as s:
        _, ab = s.residual()
    xd = torch.from_numpy(p.x0).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    J.jacobi_residual_noalloc(2, p.dims, xd.data_ptr(), None, None, out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert math.sqrt(float(out.item())) == ab


def test_noalloc_rejects_grids_beyond_its_scratch():
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(J.JacobiError) as e:
        J.jacobi_residual_noalloc(2, (1 << 16, 1 << 15), x.data_ptr(), None, None, out.data_ptr())
    assert e.value.status == J.ERR_INVALID
    assert "scratch" in J.jacobi_last_error(None)
