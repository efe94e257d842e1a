"""Failure handling on the GPU without faulting it: device allocation
failure reported as EP_ENOMEM while resident jobs keep stepping correctly;
NaN detection; errors on misuse. Failures are made on the host (an
allocator that refuses), never by faulting the device."""
import ctypes

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def test_allocation_failure_leaves_other_jobs_intact():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    L = ep.load()
    state = {"budget": 0, "live": {}}

    def alloc(nbytes, user):
        if sum(state["live"].values()) + nbytes > state["budget"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes))
        state["live"][p] = nbytes
        return p

    def free(ptr, nbytes, user):
        state["live"].pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ep.ALLOC_FN(alloc), ep.FREE_FN(free)
    h = ctypes.c_void_p()
    stream = torch.cuda.current_stream()
    assert L.ep_context_create(fa, ff, None, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)) == 0

    class Ctx(ep.Context):
        def __init__(self):
            self._h, self.jobs, self.stream, self._alloc, self._free = h, set(), stream, fa, ff
    ctx = Ctx()
    small = w.slab_case(nx=8, ny=6, nz=2)
    state["budget"] = 64 << 20
    a = ep.job_from_case(ctx, small)
    a.step(50)
    big = w.slab_case(nx=60, ny=60, nz=20, h=0.25)
    with pytest.raises(ep.EPError) as e:
        ep.job_from_case(ctx, big)
    assert e.value.code == ep.EP_ENOMEM
    a.step(50)                                # the resident job is unaffected
    ref_ctx = ep.Context()
    ref = ep.job_from_case(ref_ctx, small)
    ref.step(100)
    assert np.array_equal(a.V, ref.V)
    ref.destroy()
    ref_ctx.close()
    a.destroy()
    ctx.close()
    assert not state["live"]                  # everything handed out was returned


@pytest.mark.parametrize("variant", [6, 8])
def test_clear_error_on_a_healthy_context(variant):
    """The recovery path of a step kernel's bounded wait, exercised without
    making a wait run out: on a context whose staged (6) or fused (8) step
    variant reads its error word back after every ep_step, ep_clear_error
    synchronises and re-arms it, and the job then steps on exactly as an
    uninterrupted one."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=10, ny=6, nz=3, h=0.5)
    ctx = ep.Context()
    ep.set_cell_variant(ctx, ep.EP_FP32_MIXED, variant)
    a = ep.job_from_case(ctx, case, index_width=32)      # the staged variants read 32-bit indices
    a.step(100)
    assert a.check_finite()
    ctx.clear_error()
    a.step(100)
    b = ep.job_from_case(ctx, case, index_width=32)
    b.step(200)
    assert np.array_equal(a.V, b.V) and a.check_finite()
    ctx.close()
