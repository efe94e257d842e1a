"""The serving loop on the GPU: jobs of different sizes, models and
durations arrive while others run; each job's result in the mix equals the
same job run alone (per-cell gathers, no atomics: bitwise)."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def test_continuous_batching_results_equal_alone():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    from paper_2112_12854_b300.serving import LibBackend, Request, Server
    cases = [w.slab_case(nx=10, ny=10, nz=2, h=0.25, n_steps=300),
             w.slab_case(nx=20, ny=8, nz=3, h=0.25, D_l=0.12, n_steps=170),
             w.heart_case(h=w.heart_h_for_cells(25000, 0.25), scale=0.25, n_steps=420, av_delay=3.0),
             w.slab_case(nx=6, ny=6, nz=6, h=0.5, n_steps=95),
             w.slab_case(nx=30, ny=30, nz=2, h=0.25, n_steps=260)]
    arrivals = [0.0, 0.0, 0.05, 0.1, 0.3]
    reqs = [Request(rid=k, arrival=arrivals[k], n_steps=c.n_steps, prepare=(lambda c=c: ep.plan_from_case(c)),
                    n_cells=c.n_cells) for k, c in enumerate(cases)]
    ctx = ep.Context()
    srv = Server(LibBackend(ctx), steps_per_iter=64, workers=2)
    res = {r.rid: r for r in srv.run(reqs)}
    assert sorted(res) == list(range(len(cases)))
    assert max(x["resident"] for x in srv.log) >= 2
    for k, c in enumerate(cases):
        assert res[k].error is None
        alone = ep.job_from_case(ctx, c)
        alone.step(c.n_steps)
        assert np.array_equal(res[k].V, alone.V), k
        assert np.array_equal(res[k].act, alone.activation_times()), k
        alone.destroy()
    ctx.close()
