"""Parity at the benchmark's full size: the 9.6M-cell ventricular wedge in the
launch configuration bench.py times (autotuned cell-kernel variant, captured
graph replay, FP32 mixed; and the plain FP64 path).

The oracle cannot step 9.6M cells for hundreds of steps in a test, but the
one-step map of a cell depends only on the cells around it. We run the GPU
to step n (a wavefront is crossing the slab), take the full state, advance
the GPU one more step, and for sampled cells (random, on the front, in the
stimulus corner) run the oracle for one step on a local submesh that holds
every cell touching a node of the cell or of its face neighbours: node
values, gradients and fluxes of the sampled cell are then exact on the
submesh, so its V^{n+1} and s^{n+1} must match the GPU's."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

N_STEPS = 400


def _node_cells(tets, n_nodes):
    order = np.argsort(tets.ravel(), kind="stable")
    ptr = np.searchsorted(tets.ravel()[order], np.arange(n_nodes + 1))
    return order // 4, ptr


def _local_case(case, c, cells_of, ptr, n_cells_total):
    tets = case.tets
    touch = lambda nodes: np.unique(np.concatenate([cells_of[ptr[n]:ptr[n + 1]] for n in nodes]))
    ring = touch(tets[c])
    nb = [k for k in ring if k != c and len(np.intersect1d(tets[k], tets[c])) == 3]
    S = np.concatenate([[c], nb])
    C = touch(np.unique(tets[S].ravel()))
    nodes, inv = np.unique(tets[C].ravel(), return_inverse=True)
    sub = w.TissueCase("local", case.xyz[nodes], inv.reshape(-1, 4).astype(np.int32), case.fibre[C],
                       case.param_set[C], case.stim_mask[C], case.param_sets, case.stimuli, case.dt, 0,
                       case.threshold)
    return sub, C, int(np.flatnonzero(C == c)[0])


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_wedge_full_size_sampled_one_step(pname):
    import torch
    assert torch.cuda.is_available()
    import oracle
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    case = w.wedge_case()
    assert case.n_cells == 9_600_000
    ctx = ep.Context()
    job = ep.job_from_case(ctx, case, precision=prec)
    ep.autotune([job], 2)
    job.step(N_STEPS - job.step_index)
    assert job.step_index == N_STEPS
    nvar = 19
    snap = [job.read(v) for v in range(nvar)]
    job.step(1)
    after = [job.read(v) for v in range(nvar)]
    job.destroy()
    ctx.close()

    rng = np.random.default_rng(11)
    V = snap[0]
    front = np.flatnonzero((V > -75.0) & (V < 10.0))
    corner = np.flatnonzero(case.stim_mask > 0)
    sample = np.unique(np.concatenate([rng.choice(case.n_cells, 120, replace=False),
                                       rng.choice(front, min(120, len(front)), replace=False),
                                       rng.choice(corner, 20, replace=False)]))
    assert len(front) > 1000, "the wavefront should be crossing the slab"
    cells_of, ptr = _node_cells(case.tets, case.n_nodes)
    tolV = 1e-3 if pname == "mixed" else 1e-9
    worst = 0.0
    for c in sample:
        sub, C, loc = _local_case(case, int(c), cells_of, ptr, case.n_cells)
        s = oracle.Sim(sub)
        for v in range(nvar):
            s.set(v, snap[v][C])
        s.step_index = N_STEPS
        s.run(1)
        dv = abs(s.V[loc] - after[0][c])
        worst = max(worst, dv)
        assert dv <= tolV, (int(c), dv)
        for v in range(1, nvar):
            ref, got = s.get(v)[loc], after[v][c]
            tol = (1e-5 * max(1.0, abs(ref))) if pname == "mixed" else 1e-11 * max(1.0, abs(ref))
            assert abs(got - ref) <= tol, (int(c), v, got, ref)
    print(pname, "cells checked", len(sample), "front cells", len(front), "max |dV| one step", worst)


def test_wedge_full_size_charge_balance_fp64():
    """A property that holds at any size, checked on the full 9.6M-cell wedge
    (plain FP64, captured-graph replay): the face fluxes cancel in the
    volume-weighted sum and TP06 moves in ions the charge its V equation
    moves (stimulus carried by K+), so sum_c vol_c [C_m V - F (V_c (Na_i +
    K_i) + 2 sum volume x total calcium)] stays constant to rounding while
    the corner stimulus fires and the front spreads (300 steps)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    from test_oracle_cells import _BUF, _CM, _F, _VC
    case = w.wedge_case()
    x = case.xyz[case.tets]
    vol = np.abs(np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])) / 6.0
    del x
    ctx = ep.Context()
    job = ep.job_from_case(ctx, case, precision=ep.EP_FP64_PLAIN)
    names = ep.model_varnames(ep.EP_TP06)
    keep = ["V", "Na_i", "K_i"] + list(_BUF)
    s0 = {n: job.read(names.index(n)) for n in keep}
    job.step(300)
    s1 = {n: job.read(names.index(n)) for n in keep}
    job.destroy()
    ctx.close()
    tot = lambda c, B, K: c + B * c / (c + K)
    dq = _CM * (s1["V"] - s0["V"]) - _F * _VC * ((s1["Na_i"] - s0["Na_i"]) + (s1["K_i"] - s0["K_i"]))
    for n, (B, K, v) in _BUF.items():
        dq -= 2.0 * _F * v * (tot(s1[n], B, K) - tot(s0[n], B, K))
    swing = _CM * float(np.dot(vol, np.abs(s1["V"] - s0["V"])))
    imbalance = float(np.dot(vol, dq))
    print("charge swing", swing, "imbalance", imbalance)
    assert swing > 50.0 and abs(imbalance) < 1e-7 * swing   # measured 1.25e-9 of the swing
