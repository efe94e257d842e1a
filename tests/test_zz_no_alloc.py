"""ep_step_noalloc: the step variant for callers that must not allocate
device memory while stepping (for example a process whose device memory is
entirely reserved by another runtime's pool, or a latency-critical loop that
may not call cudaMalloc/cudaFree). It keeps the node values in the library's
static device array instead of job memory and runs the same per-cell
arithmetic as ep_step, so its results must equal ep_step's bit for bit, call
after call.

Kept in a file of its own that pytest collects last, so a run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def _three_model_slab():
    """13x7x3 cubes (1638 cells: several tiles, a ragged tail) split into
    TP06 (endo) / Courtemanche / Stewart thirds along x, fibres rotating with
    depth, two stimuli: every model region of the no-allocation kernel."""
    xyz, tets = w.kuhn_box(13, 7, 3, 0.25)
    c = w.tet_centroids(xyz, tets)
    model = np.where(c[:, 0] < 1.1, 0, np.where(c[:, 0] < 2.2, 1, 2)).astype(np.uint8)
    sets = [w.ParamSet(model=0, variant=2), w.ParamSet(model=1), w.ParamSet(model=2)]
    stim = ((c[:, 0] < 0.5).astype(np.uint8) | ((c[:, 0] > 2.9).astype(np.uint8) << 1))
    return w.TissueCase("mix", xyz, tets, w.fibres_transmural(c[:, 2], 0.0, 0.75), model, stim, sets,
                        [w.Stimulus(-52.0, 0.0, 1.0), w.Stimulus(-40.0, 5.0, 2.0)], 0.01, 0, -10.0)


CASES = {"tp06_slab": lambda: w.slab_case(nx=13, ny=9, nz=3, h=0.5),   # 2106 cells
         "three_models": _three_model_slab}


@pytest.mark.parametrize("cname", sorted(CASES))
@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_step_noalloc_equals_ep_step_two_calls(pname, cname):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    case = CASES[cname]()
    models = sorted({int(ps.model) for ps in case.param_sets})
    ctx = ep.Context()
    ref = ep.job_from_case(ctx, case, precision=prec)
    job = ep.job_from_case(ctx, case, precision=prec)
    for call in range(2):                             # two calls in a row
        ref.step(160)
        ep.step_noalloc(job, 160)
        assert job.step_index == ref.step_index == 160 * (call + 1)
        assert np.array_equal(job.V, ref.V), (call, np.abs(job.V - ref.V).max())
        for m in models:
            for var in range(1, len(ep.model_varnames(m))):
                a, b = job.read(var, model=m), ref.read(var, model=m)
                assert np.array_equal(a, b, equal_nan=True), (call, m, ep.model_varnames(m)[var])
        assert np.array_equal(job.activation_times(), ref.activation_times()), call
    assert np.isfinite(ref.activation_times()).any()
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
