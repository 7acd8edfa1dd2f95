"""Failure paths of the CUDA library, made on the host (no GPU fault, trap or
hang): non-finite inputs end a solve with JACOBI_ERR_DIVERGED, and device
allocations that fail end a create with JACOBI_ERR_OOM, release everything
taken so far, and leave the library usable."""
import numpy as np
import pytest

import oracle
from paper_2303_02543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2303_02543_gb300 import jacobi as J  # noqa: E402


def poisoned(dims, block, seed, where):
    p = inputs.make_problem(dims, block, seed, boundary="uniform", source="normal",
                            x0="uniform" if where == "x0" else "zero")
    if where == "source":
        p.source = p.source.copy()
        p.source.flat[p.source.size // 3] = np.nan
    else:
        p.x0 = p.x0.copy()
        p.x0.flat[p.x0.size // 2] = np.inf
    return p


@pytest.mark.parametrize("dtype", ["f64", "f32_refine", "bf16_refine"])
@pytest.mark.parametrize("dims,block", [((70, 50), (32, 32)), ((20, 18, 16), (8, 8, 8))])
@pytest.mark.parametrize("where", ["source", "x0"])
def test_non_finite_input_gives_diverged(dtype, dims, block, where):
    p = poisoned(dims, block, 81, where)
    with J.Solver(p.dims, p.block, dtype=dtype, faces=p.faces, source=p.source, x0=p.x0,
                  check_every=10, refine_period=10) as s:
        st, sw, rel = s.solve(1e-8, 1000)
        assert st == J.ERR_DIVERGED
        assert not np.isfinite(rel)
        assert "diverged" in J.jacobi_last_error(s.h)
    # the oracle's solve rule stops at the same check
    if dtype == "f64":
        st_o, _, sw_o, _ = oracle.solve(p.dims, p.faces, p.source, p.x0, 1e-8, 1000, 10)
    else:
        st_o, _, sw_o, _ = oracle.refine_solve(p.dims, p.faces, p.source, p.x0, 1e-8, 1000, 10,
                                               e_bf16=dtype == "bf16_refine")
    assert st_o == oracle.DIVERGED and sw == sw_o


@pytest.mark.parametrize("dtype", ["f64", "f32_refine"])
def test_diverged_problem_leaves_the_rest_of_a_batch_unchanged(dtype):
    probs = [inputs.make_problem((60, 44), (32, 16), 90 + i, boundary="uniform", source="normal", x0="zero")
             for i in range(3)]
    bad = poisoned((50, 38), (25, 19), 93, "source")
    mix = probs[:1] + [bad] + probs[1:]
    with J.Batch(mix, dtype=dtype, refine_period=10, check_every=10) as b:
        st, res = b.solve(1e-8, 10 ** 6)
        fields = [b.field(i) for i in range(len(mix))]
    assert st == J.ERR_DIVERGED
    assert res[1][0] == J.ERR_DIVERGED
    for i, p in ((0, probs[0]), (2, probs[1]), (3, probs[2])):
        assert res[i][0] == J.OK
        with J.Solver(p.dims, p.block, dtype=dtype, faces=p.faces, source=p.source, refine_period=10,
                      check_every=10) as s:
            st1, sw1, rel1 = s.solve(1e-8, 10 ** 6)
            x1 = s.field()
        assert st1 == J.OK and sw1 == res[i][1]
        assert np.array_equal(fields[i], x1)


class FailingAllocator:
    """Device allocator hooks that serve the first `fail_at - 1` requests from
    torch's caching allocator and return NULL from then on."""

    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()

        def _alloc(nbytes, stream, _user):
            self.calls += 1
            if self.calls >= self.fail_at:
                return None
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                                         stream=int(stream or 0)))
            self.live.add(ptr)
            return ptr

        def _free(ptr, _stream, _user):
            self.live.discard(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cb = (J.ALLOC_FN(_alloc), J.FREE_FN(_free))

    def __enter__(self):
        J.load().jacobi_set_allocator(self.cb[0], self.cb[1], None)
        return self

    def __exit__(self, *exc):
        J.use_torch_allocator(True)
        return False


@pytest.mark.parametrize("fail_at", [1, 2, 4, 6, 9, 13, 18, 24])
def test_failed_allocation_gives_oom_and_releases_everything(fail_at):
    p = inputs.make_problem((130, 70), (64, 32), 95, boundary="uniform", source="normal", x0="uniform")
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with FailingAllocator(fail_at) as fa:
        with pytest.raises(J.JacobiError) as e:
            J.Solver(p.dims, p.block, dtype="f32_refine", faces=p.faces, source=p.source, x0=p.x0,
                     torch_alloc=False)
        assert e.value.status == J.ERR_OOM
        assert fa.calls == fail_at
        assert not fa.live, "a failed create kept device memory"
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    # the library works normally afterwards
    with J.Solver(p.dims, p.block, faces=p.faces, source=p.source, x0=p.x0) as s:
        s.sweep(7)
        x = s.field()
    assert np.array_equal(x, oracle.sweeps(p.dims, p.faces, p.source, p.x0, 7))


@pytest.mark.parametrize("fail_at", [1, 3, 8, 20, 40])
def test_failed_allocation_in_a_batch_gives_oom(fail_at):
    probs = [inputs.make_problem((40 + 10 * i, 30), (16, 16), 96 + i, boundary="uniform", source="normal",
                                 x0="zero") for i in range(3)]
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with FailingAllocator(fail_at) as fa:
        with pytest.raises(J.JacobiError) as e:
            J.Batch(probs, dtype="f32_refine", torch_alloc=False)
        assert e.value.status == J.ERR_OOM
        assert not fa.live
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    with J.Batch(probs, dtype="f32_refine") as b:
        st, res = b.solve(1e-8, 10 ** 6)
    assert st == J.OK


def test_failed_arena_allocation_gives_oom_at_server_create():
    with FailingAllocator(1) as fa:
        with pytest.raises(J.JacobiError) as e:
            J.Server("f32_refine", budget_bytes=64 << 20, max_slots=4, torch_alloc=False)
        assert e.value.status == J.ERR_OOM
        assert fa.calls == 1
    p = inputs.make_problem((48, 40), (16, 16), 97, boundary="uniform", source="normal", x0="zero")
    with J.Server("f32_refine", budget_bytes=64 << 20, max_slots=4) as srv:
        t = srv.submit(p, 1e-8, 10 ** 6)
        assert srv.wait(t, 120.0)
        st, sw, rel, _, x = srv.poll(t)
    assert st == J.OK and rel <= 1e-8
    assert oracle.relative_residual(p.dims, p.faces, p.source, x) <= 1e-8
