"""Parity of the CUDA path on jobs with a 2D Purkinje shell (triangles folded
into the same per-cell coefficients as the tets, Sec. 2 / 3.2) with the FP64
oracle's edge-by-edge shell operator, through the C ABI: a shell-only
Stewart strip (front speed, Table 2), and a tet slab beside a shell that a
conduction-graph cable excites through a triggered junction."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu

D_PURK = 3.95 / 1.4


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    c = ep.Context()
    yield c
    c.close()


def _prec(name):
    from paper_2112_12854_b300 import ep
    return ep.EP_FP32_MIXED if name == "mixed" else ep.EP_FP64_PLAIN


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_shell_strip_parity_and_speed(ctx, pname):
    import oracle
    from paper_2112_12854_b300 import ep
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    h, dt = 0.2, 0.001
    xyz, tris = w.tri_box(100, 3, h)
    n = len(tris)
    c = w.tri_centroids(xyz, tris)
    case = w.TissueCase("shell", xyz, np.zeros((0, 4), np.int32), w.fibres_uniform(n), np.zeros(n, np.uint8),
                        (c[:, 0] < 1.0).astype(np.uint8), [w.ParamSet(model=2, D_l=D_PURK, D_t=D_PURK)],
                        [w.Stimulus(-100.0, 0.0, 1.0)], dt, 0, 0.0, tris=tris)
    o = oracle.Sim(case)
    j = ep.job_from_case(ctx, case, precision=prec)
    assert j.n_cells == n
    done = 0
    for k in (1500, 4000, 7000):
        o.run(k - done)
        j.step(k - done)
        done = k
        assert np.abs(j.V - o.V).max() <= tv
    a = j.activation_times()
    assert act_error(a, o.activation_times()) <= ta
    sel = (c[:, 0] > 5) & (c[:, 0] < 15)
    cv = np.polyfit(a[sel], c[sel, 0], 1)[0]
    print(pname, "shell front speed", cv)
    assert abs(cv - 4.0) < 0.4
    j.destroy()


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_tets_shell_and_graph_junction(ctx, pname):
    import oracle
    from paper_2112_12854_b300 import ep
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    xyz_t, tets = w.kuhn_box(8, 4, 2, 0.25)
    # shell squares of 0.4 mm allow dt = 0.004 ms (explicit bound dt rho < 2); much smaller
    # steps make V's FP32 increments approach its rounding step at rest
    xyz_s, tris = w.tri_box(20, 2, 0.4, origin=(0.0, 0.0, 3.0))
    xyz = np.concatenate([xyz_t, xyz_s])
    tris = tris + len(xyz_t)
    nt, ns = len(tets), len(tris)
    ct = w.tet_centroids(xyz_t, tets)
    cs = w.tri_centroids(xyz, tris)
    ps = np.concatenate([np.zeros(nt, np.uint8), np.ones(ns, np.uint8)])
    sm = np.concatenate([(ct[:, 0] < 0.5).astype(np.uint8), np.zeros(ns, np.uint8)])
    case = w.TissueCase("mixed", xyz, tets, w.fibres_uniform(nt + ns), ps, sm,
                        [w.ParamSet(model=0), w.ParamSet(model=2, D_l=D_PURK, D_t=D_PURK), w.ParamSet(model=2)],
                        [w.Stimulus(-100.0, 0.0, 1.0)], 0.004, 0, 0.0, tris=tris)
    g = w.chain_graph(20, 0.2, start=(-4.0, 0.2, 3.0), param_set=2, stim_nodes=3,
                      params=w.GraphParams(radius=0.5, amplitude=-300.0, duration=1.0))
    g.junction_node = np.array([19], np.int32)
    g.junction_cell = np.array([nt + int(np.argmin(np.linalg.norm(cs - g.xyz[19], axis=1)))], np.int32)
    g.junction_mode = np.array([w.JUNC_TRIGGERED], np.uint8)
    o = oracle.Sim(case)
    o.attach_graph(g)
    j = ep.job_from_case(ctx, case, precision=prec)
    j.attach_graph(g, node_model=np.full(20, 2, np.uint8))
    done = 0
    for k in (750, 2000, 3000):
        o.run(k - done)
        j.step(k - done)
        done = k
        dv = np.abs(j.V - o.V)
        print(pname, k, "max|dV| tets", dv[:nt].max(), "shell", dv[nt:].max())
        assert dv.max() <= tv
        assert np.abs(j.graph_read(0, model=2) - o.graph_get(0)).max() <= tv
    a = j.activation_times()
    assert act_error(a, o.activation_times()) <= ta
    assert np.isfinite(a[nt:]).mean() > 0.9 and np.isfinite(a[:nt]).any()
    with pytest.raises(ep.EPError):
        j.enable_bidomain(0.3, 0.1)                 # the shell is a monodomain medium
    j.destroy()


@pytest.mark.parametrize("pname,two_way", [("mixed", 0), ("plain", 0), ("mixed", 1)])
def test_cell_communication_nodes(ctx, pname, two_way):
    """Communication nodes between shell cells and myocardial cells (Sec.
    3.3, EP_PMJ_CELL, a graph without nodes): the shell's front excites the
    slab through them after the orthodromic delay; with two-way coupling a
    stimulated slab excites the shell back. V and activation times against
    the oracle."""
    import oracle
    from paper_2112_12854_b300 import ep
    from test_oracle_shell import _shell_and_slab
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    dt = 0.004
    case, nt, ct, cs = _shell_and_slab(dt, stim_shell=not two_way, stim_slab=bool(two_way))
    src = nt + np.array([int(np.argmin(np.linalg.norm(cs - p, axis=1))) for p in ([-0.3, 0.4, 0.25], [-3.0, 0.2, 0.25])])
    dst = np.array([int(np.argmin(np.linalg.norm(ct - p, axis=1))) for p in ([0.2, 0.5, 0.25], [1.5, 0.5, 0.25])])
    gp = w.GraphParams(delay_ortho=5.0, delay_anti=3.0, amplitude=-300.0, duration=1.0, radius=0.3,
                       two_way=two_way)
    g = w.Graph(np.zeros((0, 3)), np.zeros((0, 2), np.int32), np.zeros(0, np.uint8), np.zeros(0, np.uint8),
                src.astype(np.int32), dst.astype(np.int32), np.full(2, w.JUNC_CELL, np.uint8), gp)
    o = oracle.Sim(case)
    o.attach_graph(g)
    j = ep.job_from_case(ctx, case, precision=prec)
    j.attach_graph(g, node_model=np.zeros(0, np.uint8))
    done = 0
    for k in (1500, 3000, 4000):
        o.run(k - done)
        j.step(k - done)
        done = k
        assert np.abs(j.V - o.V).max() <= tv
    a, ao = j.activation_times(), o.activation_times()
    assert act_error(a, ao) <= ta
    if two_way:
        assert np.isfinite(ao[nt:]).mean() > 0.9 and ao[src[0]] > ao[dst[0]] + gp.delay_anti
    else:
        assert np.isfinite(ao[:nt]).mean() > 0.9 and np.nanmin(ao[:nt]) > ao[src].min() + gp.delay_ortho
    j.destroy()
