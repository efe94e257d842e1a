"""Parity of the CUDA conduction-graph path (graph reaction + subcycled
vertex FV diffusion + junctions) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu

PRECISIONS = ["mixed", "plain"]


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


def _slab(dt=0.02, cubes=(12, 4, 2), stim=False):
    xyz, tets = w.kuhn_box(*cubes, 0.25, origin=(0.0, 0.0, -1.0))
    n = tets.shape[0]
    c = w.tet_centroids(xyz, tets)
    sm = (c[:, 0] < 0.5).astype(np.uint8) if stim else np.zeros(n, np.uint8)
    return w.TissueCase("slab", xyz, tets, w.fibres_uniform(n), np.zeros(n, np.uint8), sm,
                        [w.ParamSet(model=0), w.ParamSet(model=2), w.ParamSet(model=1)],
                        [w.Stimulus(-100.0, 0.0, 2.0)], dt, 0, -20.0)


def _tree(rng, n_seg=12, seg_nodes=8, ds=0.2, origin=(0.0, 0.5, 0.3)):
    """A small branched tree: segments of seg_nodes nodes, each new segment
    starting from the end of a random earlier one (branch nodes of degree 3+)."""
    xyz = [np.asarray(origin, float)]
    edges, ends = [], [0]
    for s in range(n_seg):
        start = ends[rng.integers(0, len(ends))]
        d = rng.standard_normal(3)
        d[2] *= 0.2
        d /= np.linalg.norm(d)
        prev = start
        for k in range(seg_nodes):
            xyz.append(xyz[prev] + ds * d)
            edges.append((prev, len(xyz) - 1))
            prev = len(xyz) - 1
        ends.append(prev)
    return np.array(xyz), np.array(edges, np.int32), ends


def _run_both(ctx, case, graph, prec, outs, node_model):
    import oracle
    from paper_2112_12854_b300 import ep
    o = oracle.Sim(case)
    o.attach_graph(graph)
    j = ep.job_from_case(ctx, case, precision=prec)
    j.attach_graph(graph, node_model=node_model)
    assert j.graph_info()["substeps"] == o.graph_substeps
    res = []
    done = 0
    for n in outs:
        o.run(n - done)
        j.step(n - done)
        done = n
        res.append((o.V, j.V, o.graph_get(0), j.graph_read(0, model=int(node_model[0]))))
    return o, j, res


@pytest.mark.parametrize("pname", PRECISIONS)
def test_purkinje_cable_alone(ctx, pname):
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    case = _slab()
    g = w.chain_graph(60, 0.2, start=(0.0, 2.0, 0.5), param_set=1, stim_nodes=10)
    nm = np.full(60, 2, np.uint8)
    o, j, res = _run_both(ctx, case, g, prec, [100, 400, 800], nm)
    for ov, jv, og, jg in res:
        assert np.abs(jg - og).max() <= tv and np.abs(jv - ov).max() <= tv
    assert act_error(j.graph_activation_times(), o.graph_activation_times()) <= ta
    j.destroy()


@pytest.mark.parametrize("pname", PRECISIONS)
@pytest.mark.parametrize("mode", ["resistive", "triggered"])
def test_tree_with_junctions(ctx, pname, mode):
    """A branched Stewart tree stimulated at its root, coupled at its branch
    ends to slab cells: resistive PMJs, or triggered two-way junctions with a
    radius (orthodromic and antidromic delays)."""
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    rng = np.random.default_rng(5)
    case = _slab(cubes=(16, 8, 3))
    xyz, edges, ends = _tree(rng)
    n = xyz.shape[0]
    cen = w.tet_centroids(case.xyz, case.tets)
    jn = np.array(ends[1:], np.int32)
    jc = np.array([np.argmin(np.linalg.norm(cen - xyz[e], axis=1)) for e in jn], np.int32)
    # a junction drives one myocardial cell against its neighbours' sink: the resistive
    # coupling rate must be large enough to excite it (dt * g_cell = 0.08 stays explicit-stable)
    gp = w.GraphParams(g_graph=0.3, g_cell=4.0, radius=0.3, two_way=1, delay_ortho=2.0, delay_anti=1.5,
                       amplitude=-80.0, duration=1.0)
    sm = np.zeros(n, np.uint8)
    sm[:6] = 1
    jm = np.full(jn.size, w.JUNC_RESISTIVE if mode == "resistive" else w.JUNC_TRIGGERED, np.uint8)
    g = w.Graph(xyz, edges, np.ones(n, np.uint8), sm, jn, jc, jm, gp)
    o, j, res = _run_both(ctx, case, g, prec, [150, 500, 1000], np.full(n, 2, np.uint8))
    for ov, jv, og, jg in res:
        assert np.abs(jg - og).max() <= tv, np.abs(jg - og).max()
        assert np.abs(jv - ov).max() <= tv, np.abs(jv - ov).max()
    assert act_error(j.activation_times(), o.activation_times()) <= ta
    assert act_error(j.graph_activation_times(), o.graph_activation_times()) <= ta
    assert np.isfinite(o.activation_times()).sum() > 20       # the myocardium was reached through the junctions
    j.destroy()


def test_graph_jobs_batched_bitwise(ctx):
    """Graph jobs in a batch with graph-less jobs and with each other give the
    results they give alone (mixed models on the graph: Courtemanche bundle
    into a Stewart tree, per-edge diffusivities)."""
    from paper_2112_12854_b300 import ep
    rng = np.random.default_rng(9)
    case = _slab(cubes=(10, 6, 2))
    xyz, edges, ends = _tree(rng, n_seg=6)
    n = xyz.shape[0]
    ps = np.ones(n, np.uint8)
    ps[: n // 3] = 2                                   # Courtemanche nodes
    nm = np.where(ps == 2, 1, 2).astype(np.uint8)
    cen = w.tet_centroids(case.xyz, case.tets)
    jn = np.array(ends[1:3], np.int32)
    jc = np.array([np.argmin(np.linalg.norm(cen - xyz[e], axis=1)) for e in jn], np.int32)
    edD = rng.uniform(0.5, 2.5, edges.shape[0])
    sm = np.zeros(n, np.uint8)
    sm[:4] = 1
    g = w.Graph(xyz, edges, ps, sm, jn, jc, np.zeros(2, np.uint8), w.GraphParams(), edge_D=edD)

    def make():
        j = ep.job_from_case(ctx, case)
        j.attach_graph(g, node_model=nm)
        return j
    alone = make()
    alone.step(300)
    a1, a2 = make(), make()
    other = ep.job_from_case(ctx, w.slab_case(nx=7, ny=5, nz=2))
    ep.step([other, a1, a2], 300)
    for j in (a1, a2):
        assert np.array_equal(j.V, alone.V)
        assert np.array_equal(j.graph_read(0, model=1), alone.graph_read(0, model=1))
    for j in (alone, a1, a2, other):
        j.destroy()


@pytest.mark.parametrize("pname", PRECISIONS)
def test_graph_substeps_one_launch_equals_launches(pname):
    """All diffusion substeps of a step in one launch (each block on a tile
    of graph nodes and its neighbourhood in shared memory) give bitwise the
    results of one launch per substep: the quarter-scale whole heart with its
    conduction system (trees, bundles, resistive and triggered junctions),
    batched with a branched-tree slab job whose graph has a different
    substep count, over 3000 steps (the front through the graph and into the
    ventricles)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    prec = _prec(pname)
    case, g = w.whole_heart(h=w.heart_h_for_cells(25000, 0.25), scale=0.25, n_tree=1500, n_pmj=150)
    node_model = np.array([ps.model for ps in case.param_sets], np.uint8)[g.param_set]
    rng = np.random.default_rng(3)
    xyz, edges, ends = _tree(rng)
    slab = _slab(dt=0.01, stim=True)
    c = w.tet_centroids(slab.xyz, slab.tets)
    sm = np.zeros(len(xyz), np.uint8)
    sm[:6] = 1
    jn = np.array(ends[1:4], np.int32)
    jc = np.array([int(np.argmin(np.linalg.norm(c - xyz[e], axis=1))) for e in jn], np.int32)
    tg = w.Graph(xyz, edges, np.ones(len(xyz), np.uint8), sm, jn, jc, np.full(3, w.JUNC_RESISTIVE, np.uint8),
                 w.GraphParams(g_cell=4.0))
    out = []
    for mode in (ep.EP_GRAPH_SUBSTEPS_LAUNCHES, ep.EP_GRAPH_SUBSTEPS_LOCAL):
        ctx = ep.Context()
        ctx.set_graph_kernel(mode)
        a = ep.job_from_case(ctx, case, precision=prec)
        a.attach_graph(g, node_model=node_model)
        b = ep.job_from_case(ctx, slab, precision=prec)
        b.attach_graph(tg, node_model=np.full(len(xyz), 2, np.uint8))
        assert a.graph_info()["substeps"] != b.graph_info()["substeps"]
        ep.step([a, b], 3000)
        res = []
        for j in (a, b):
            res += [j.V, j.activation_times(), j.graph_activation_times()]
            res += [j.graph_read(k, model=m) for m in (1, 2) for k in range(len(ep.model_varnames(m)))]
        out.append(res)
        ctx.close()
    for x, y in zip(*out):
        assert np.array_equal(x, y, equal_nan=True)
    assert np.isfinite(out[0][2]).any()
