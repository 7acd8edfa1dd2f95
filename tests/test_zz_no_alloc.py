"""The allocation-free residual entry point, through the C ABI.

jacobi_residual_noalloc serves callers that cannot call cudaMalloc (device
memory owned in full by another runtime, or loops that must never stall the
device on an allocation).  Its scratch is a fixed device array inside the
library.  This file is named so that pytest collects it last; it must pass
alone in a fresh process and after every other test.
"""
import ctypes
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
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
            # and against the oracle's residual of the same field
            ref_o, _ = oracle.residual(p.dims, p.faces, p.source, s.field())
            assert abs(got - ref_o) <= 1e-12 * ref_o
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


def test_noalloc_makes_no_device_allocation():
    """The defining property: no call of the entry point reaches an allocator.
    A counting allocator registered with jacobi_set_allocator sees no call,
    and neither torch's allocated bytes nor the device's free memory move
    across repeated calls once the first call has run (the first call in a
    context may load the library's module, which holds the fixed scratch)."""
    lib = J.load()
    p = inputs.make_problem((200, 150), (200, 150), 63, boundary="uniform", source="normal", x0="uniform")
    xd, fd, faces = device_inputs(p, p.x0)
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, user):
        calls["alloc"] += 1
        return None  # a failed allocation: any use would surface as an error

    def _free(ptr, stream, user):
        calls["free"] += 1

    a_cb, f_cb = J.ALLOC_FN(_alloc), J.FREE_FN(_free)
    lib.jacobi_set_allocator(a_cb, f_cb, None)
    try:
        first = noalloc_rss(p, xd, fd, faces)
        torch.cuda.synchronize()
        alloc0 = torch.cuda.memory_allocated()
        free0, _ = torch.cuda.mem_get_info()
        vals = [noalloc_rss(p, xd, fd, faces) for _ in range(5)]
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == alloc0
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        J.use_torch_allocator(True)  # the binding's hooks for the tests that follow
    assert calls == {"alloc": 0, "free": 0}
    assert all(v == first for v in vals)
    ref, _ = oracle.residual(p.dims, p.faces, p.source, p.x0)
    assert abs(first - ref) <= 1e-12 * ref


_CONTEXTS_SCRIPT = textwrap.dedent("""
    import ctypes, sys
    import numpy as np
    sys.path.insert(0, sys.argv[1])
    import oracle
    from paper_2303_02543_gb300 import inputs
    from paper_2303_02543_gb300 import jacobi as J

    cu = ctypes.CDLL("libcuda.so.1")
    u64 = ctypes.c_uint64

    def ck(r, what):
        if r != 0:
            raise SystemExit(f"{what} returned {r}")

    def residual_in_current_context(seed, dims):
        # device buffers of the current context, the field and inputs copied in
        p = inputs.make_problem(dims, dims, seed, boundary="uniform", source="normal", x0="uniform")
        bufs = []

        def dev(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            d = u64()
            ck(cu.cuMemAlloc_v2(ctypes.byref(d), ctypes.c_size_t(a.nbytes)), "cuMemAlloc")
            ck(cu.cuMemcpyHtoD_v2(d, a.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(a.nbytes)), "cuMemcpyHtoD")
            bufs.append(d)
            return d.value

        x, f = dev(p.x0), dev(p.source)
        faces = [dev(g) for g in p.faces]
        out = dev(np.full(1, np.nan))
        J.jacobi_residual_noalloc(p.ndim, p.dims, x, f, faces, out, None)
        ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
        got = np.zeros(1)
        ck(cu.cuMemcpyDtoH_v2(got.ctypes.data_as(ctypes.c_void_p), u64(out), ctypes.c_size_t(8)), "cuMemcpyDtoH")
        for d in bufs:
            ck(cu.cuMemFree_v2(d), "cuMemFree")
        ref, _ = oracle.residual(p.dims, p.faces, p.source, p.x0)
        if not abs(got[0] - ref) <= 1e-12 * ref:
            raise SystemExit(f"seed {seed}: noalloc {got[0]!r} vs oracle {ref!r}")

    ck(cu.cuInit(0), "cuInit")
    dev = ctypes.c_int()
    ck(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
    prim = ctypes.c_void_p()
    ck(cu.cuDevicePrimaryCtxRetain(ctypes.byref(prim), dev), "cuDevicePrimaryCtxRetain")
    ck(cu.cuCtxSetCurrent(prim), "cuCtxSetCurrent(primary)")
    residual_in_current_context(71, (300, 90))
    # a second context of the same device, made current through the driver API
    ctx2 = ctypes.c_void_p()
    if hasattr(cu, "cuCtxCreate_v4"):
        ck(cu.cuCtxCreate_v4(ctypes.byref(ctx2), None, 0, dev), "cuCtxCreate")
    else:
        ck(cu.cuCtxCreate_v2(ctypes.byref(ctx2), 0, dev), "cuCtxCreate")
    ck(cu.cuCtxSetCurrent(ctx2), "cuCtxSetCurrent(second)")
    residual_in_current_context(72, (150, 60, 20))
    residual_in_current_context(73, (300, 90))
    ck(cu.cuCtxSetCurrent(prim), "cuCtxSetCurrent(primary again)")
    residual_in_current_context(74, (150, 60, 20))
    ck(cu.cuCtxDestroy_v2(ctx2), "cuCtxDestroy")
    residual_in_current_context(75, (300, 90))
    ck(cu.cuDevicePrimaryCtxRelease_v2(dev), "cuDevicePrimaryCtxRelease")
    print("contexts ok")
""")


def test_noalloc_follows_the_current_context():
    """The scratch array has one instance per CUDA context, so its address is
    looked up per context: calls in the primary context, in a second context
    of the same device made current through the driver API (a caller whose
    memory another runtime owns), and back in the primary context all give the
    oracle's residual.  Runs in a fresh process without torch, which would
    otherwise own the primary context."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CONTEXTS_SCRIPT, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "contexts ok" in r.stdout
