"""Parity of the CUDA second-order Adams-Bashforth option for the
non-gating variables (Sec. 4) with the FP64 oracle's AB2, through the C ABI:
a slab with TP06, Courtemanche and Stewart regions; a checkpoint written
back mid-run restarts the history on both sides (one forward-Euler step);
and an AB2 job in a batch with forward-Euler jobs gives its results alone."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    c = ep.Context()
    yield c
    c.close()


def _slab(cubes=(12, 8, 3), h=0.25, dt=0.01):
    # AB2's explicit stability interval is half forward Euler's: dt rho(L) < 1
    xyz, tets = w.kuhn_box(*cubes, h)
    n = tets.shape[0]
    c = w.tet_centroids(xyz, tets)
    ps = (np.arange(n) * 3 // n).astype(np.uint8)
    sets = [w.ParamSet(model=0, variant=2), w.ParamSet(model=1), w.ParamSet(model=2)]
    return w.TissueCase("slab", xyz, tets, w.fibres_transmural(c[:, 2], 0.0, cubes[2] * h), ps,
                        (c[:, 0] < 0.6).astype(np.uint8), sets, [w.Stimulus(-80.0, 0.0, 1.0)], dt, 0, -20.0)


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_ab2_parity_and_restart(ctx, pname):
    import oracle
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    tv, ta = tolerances(prec)
    case = _slab()
    o = oracle.Sim(case)
    o.set_integrator(1)
    j = ep.job_from_case(ctx, case, precision=prec, integrator=ep.EP_INTEGRATOR_AB2)
    fe = ep.job_from_case(ctx, case, precision=prec)           # forward Euler, for contrast
    done = 0
    for n in (300, 800):
        o.run(n - done)
        j.step(n - done)
        fe.step(n - done)
        done = n
        dv = np.abs(j.V - o.V).max()
        print(pname, n, "AB2 max|dV|", dv, "FE vs AB2", np.abs(fe.V - o.V).max())
        assert dv <= tv
    if pname == "plain":
        assert np.abs(fe.V - o.V).max() > 1e3 * tv             # AB2 is not forward Euler
    # checkpoint written back: each side restarts its history with one FE step
    for m, names in ((0, None), (1, None), (2, None)):
        nv = len(ep.model_varnames(m))
        for v in range(1 if m else 0, nv):
            vals = j.read(v, model=m)
            sel = ~np.isnan(vals)
            full = o.get(v)
            full[sel] = vals[sel]
            o.set(v, full)
            j.write(v, vals, model=m)
    o.run(400)
    j.step(400)
    dv = np.abs(j.V - o.V).max()
    print(pname, "after restart max|dV|", dv)
    assert dv <= tv
    assert act_error(j.activation_times(), o.activation_times()) <= ta
    j.destroy()
    fe.destroy()


def test_ab2_batched_with_forward_euler_jobs(ctx):
    from paper_2112_12854_b300 import ep
    case = _slab(cubes=(8, 6, 2))
    alone = ep.job_from_case(ctx, case, integrator=ep.EP_INTEGRATOR_AB2)
    alone.step(600)
    a1 = ep.job_from_case(ctx, case, integrator=ep.EP_INTEGRATOR_AB2)
    f1 = ep.job_from_case(ctx, case)
    f_alone = ep.job_from_case(ctx, case)
    f_alone.step(600)
    ep.step([f1, a1], 600)
    assert np.array_equal(a1.V, alone.V)
    assert np.array_equal(f1.V, f_alone.V)
    for x in (alone, a1, f1, f_alone):
        x.destroy()
