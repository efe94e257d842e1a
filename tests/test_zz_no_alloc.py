"""ep_step_noalloc: the step variant for callers that must not allocate
device memory while stepping (for example a process whose device memory is
entirely reserved by another runtime's pool, or a latency-critical loop that
may not call cudaMalloc/cudaFree). It keeps the node values in the library's
static device array instead of job memory; its results must equal those of
ep_step on the same inputs, call after call.

Kept in a file of its own that pytest collects last, so a run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

import workloads as w
from gpu_common import tolerances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_step_noalloc_matches_ep_step_two_calls(pname):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    tv, ta = tolerances(prec)
    case = w.slab_case(nx=13, ny=9, nz=3, h=0.5)      # 2106 cells: several tiles and a ragged tail
    ctx = ep.Context()
    ref = ep.job_from_case(ctx, case, precision=prec)
    job = ep.job_from_case(ctx, case, precision=prec)
    for call in range(2):                             # two calls in a row
        ref.step(160)
        ep.step_noalloc(job, 160)
        assert job.step_index == ref.step_index == 160 * (call + 1)
        dv = np.abs(job.V - ref.V).max()
        assert dv <= tv, (call, dv)
        for var in range(1, 19):
            a, b = job.read(var), ref.read(var)
            assert np.abs(a - b).max() <= tv * max(1.0, np.abs(b).max()), (call, var)
        a, b = job.activation_times(), ref.activation_times()
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        if fin.any():
            assert np.abs(a[fin] - b[fin]).max() <= ta
    ref.destroy()
    job.destroy()
    ctx.close()


def test_step_noalloc_rejects_meshes_over_the_limit():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_12854_b300 import ep
    # one tet over a node array one entry longer than the limit (unused nodes
    # are allowed): rejected before any launch
    xyz = np.zeros((ep.NOALLOC_MAX_NODES + 1, 3))
    xyz[1:4] = np.eye(3)
    ctx = ep.Context()
    j = ctx.mesh(xyz, np.array([[0, 1, 2, 3]], np.int32))
    j.set_params(ep.make_params(0.02, [w.ParamSet()]))
    with pytest.raises(ep.EPError) as e:
        ep.step_noalloc(j, 1)
    assert e.value.code == ep.EP_EINVAL and "at most" in str(e.value)
    j.destroy()
    ctx.close()
