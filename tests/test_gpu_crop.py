"""Parity over a beat's first 25 ms on the 1.2M-cell crop of the benchmark
wedge (100 x 100 x 20 cubes of 0.25 mm, the wedge's construction: TP06
endo / M / epi by depth, fibres rotating -60..+60 deg, corner stimulus):
FP32 mixed and FP64 plain against one oracle run, V at every cell every
5 ms, the activation map and every state variable at the end."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu


def test_wedge_crop_every_5ms():
    import torch
    assert torch.cuda.is_available()
    import oracle
    from paper_2112_12854_b300 import ep
    case = w.wedge_case(nx=100, ny=100, nz=20, h=0.25, n_steps=1250)
    assert case.n_cells == 1_200_000
    ctx = ep.Context()
    jobs = {p: ep.job_from_case(ctx, case, precision=p) for p in (ep.EP_FP32_MIXED, ep.EP_FP64_PLAIN)}
    o = oracle.Sim(case)
    done = 0
    for k in range(250, 1251, 250):
        o.run(k - done)
        for j in jobs.values():
            j.step(k - done)
        done = k
        ref = o.V
        for p, j in jobs.items():
            tv, _ = tolerances(p)
            err = np.abs(j.V - ref).max()
            print(k * case.dt, "ms", "mixed" if p == ep.EP_FP32_MIXED else "plain", "max|dV|", err)
            assert err <= tv
    a = o.activation_times()
    assert np.isfinite(a).sum() > 10000                      # the front has crossed a good part of the crop
    t_end = 1250 * case.dt
    for p, j in jobs.items():
        _, ta = tolerances(p)
        g = j.activation_times()
        # cells crossing within the last 0.1 ms may fall on either side of the final step
        settled = (np.where(np.isfinite(a), a, np.inf) < t_end - 0.1) | (np.where(np.isfinite(g), g, np.inf) < t_end - 0.1)
        assert act_error(g[settled], a[settled]) <= ta
        # every TP06 state variable at 25 ms, relative to its largest magnitude on the crop
        rel_tol = 1e-9 if p == ep.EP_FP64_PLAIN else 1e-3
        for v, name in enumerate(ep.model_varnames(ep.EP_TP06)):
            if v == 0:
                continue
            r = o.get(v)
            rel = np.abs(j.read(v) - r).max() / np.abs(r).max()
            print("mixed" if p == ep.EP_FP32_MIXED else "plain", f"{name:>6s} max|d|/max|ref| {rel:.2e}")
            assert rel <= rel_tol, name
        j.destroy()
    ctx.close()
