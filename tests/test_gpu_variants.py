"""The cell kernel's launch-shape variants (ep_autotune / ep_set_cell_variant)
change only the launch configuration: every variant must give bitwise the
same state, and the autotuner's steps are ordinary time steps."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_all_cell_variants_bitwise_identical(pname):
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    case = w.slab_case(nx=11, ny=7, nz=3, h=0.5)
    ctx = ep.Context()
    ref = None
    for v in range(ep.N_CELL_VARIANTS):
        ep.set_cell_variant(ctx, prec, v)
        j = ep.job_from_case(ctx, case, precision=prec)
        j.step(120)
        state = [j.read(k) for k in range(19)] + [j.activation_times()]
        if ref is None:
            ref = state
        else:
            for a, b in zip(state, ref):
                assert np.array_equal(a, b, equal_nan=True), v
        j.destroy()
    ctx.close()


def test_autotune_steps_are_real_steps():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=9, ny=6, nz=3, h=0.5)
    ctx = ep.Context()
    a = ep.job_from_case(ctx, case)
    chosen, ms = ep.autotune([a], 4)
    assert 0 <= chosen[0] < ep.N_CELL_VARIANTS and chosen[1] == -1
    assert np.all(ms[0] > 0)
    assert a.step_index == 4 * ep.N_CELL_VARIANTS
    a.step(50)
    b = ep.job_from_case(ctx, case)
    b.step(4 * ep.N_CELL_VARIANTS + 50)
    assert np.array_equal(a.V, b.V)
    ctx.close()
