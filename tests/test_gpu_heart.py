"""Whole-heart topology with its conduction system (atrial bundle, AV delay
line, Purkinje trees, resistive PMJs, triggered atrial communication nodes)
at 1/4 scale: the CUDA path against the FP64 oracle over the first 200 ms
of a beat (sinus node -> atria -> AV delay -> His -> Purkinje -> ventricles)."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_whole_heart_quarter_scale(pname):
    import torch
    assert torch.cuda.is_available()
    import oracle
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    tv, ta = tolerances(prec)
    case, g = w.whole_heart(h=w.heart_h_for_cells(25000, 0.25), scale=0.25, n_tree=1500, n_pmj=150)
    node_model = np.array([ps.model for ps in case.param_sets], np.uint8)[g.param_set]
    o = oracle.Sim(case)
    o.attach_graph(g)
    ctx = ep.Context()
    j = ep.job_from_case(ctx, case, precision=prec)
    j.attach_graph(g, node_model=node_model)
    done = 0
    worst = 0.0
    for n in (2500, 5000, 7500, 10000):
        o.run(n - done)
        j.step(n - done)
        done = n
        worst = max(worst, np.abs(j.V - o.V).max(), np.abs(j.graph_read(0) - o.graph_get(0)).max())
    print(pname, "whole heart max |dV|", worst)
    assert worst <= tv
    a = o.activation_times()
    assert act_error(j.activation_times(), a) <= ta
    assert act_error(j.graph_activation_times(), o.graph_activation_times()) <= ta
    # the activation reached both atria and the ventricles within the 200 ms
    atr = case.param_set == 2
    assert np.isfinite(a[atr]).mean() > 0.9 and np.isfinite(a[~atr]).mean() > 0.5
    ctx.close()
