"""Pins of the oracle's conduction graph (vertex-based 1D FV, Sec. 3.2) and
of its junctions with the myocardium (Sec. 3.3)."""
import os

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return {k: float(v) for k, v in rows}


def _tet_case(dt=0.02, amp=-100.0, dur=2.0, n_cubes=None):
    if n_cubes is None:
        xyz = np.array([[0, 0, -5], [0.5, 0, -5], [0, 0.5, -5], [0, 0, -4.5]], float)
        tets = np.array([[0, 1, 2, 3]], np.int32)
    else:
        xyz, tets = w.kuhn_box(*n_cubes, 0.25, origin=(0.0, 0.0, -5.0))
    n = tets.shape[0]
    return w.TissueCase("tet", xyz, tets, w.fibres_uniform(n), np.zeros(n, np.uint8), np.zeros(n, np.uint8),
                        [w.ParamSet(model=0), w.ParamSet(model=2)], [w.Stimulus(amp, 0.0, dur)], dt, 0, -20.0)


def _random_tree(n, rng):
    parent = np.array([rng.integers(0, i) for i in range(1, n)])
    edges = np.stack([parent, np.arange(1, n)], axis=1).astype(np.int32)
    xyz = np.zeros((n, 3))
    for i in range(1, n):
        d = rng.standard_normal(3)
        xyz[i] = xyz[parent[i - 1]] + rng.uniform(0.1, 0.5) * d / np.linalg.norm(d)
    return xyz, edges


def test_chain_laplacian_is_three_point_stencil(orc):
    """On a uniform cable the vertex FV operator is D (W_{i+1} - 2 W_i + W_{i-1}) / ds^2
    inside and 2 D (W_1 - W_0) / ds^2 at a free end (half control length)."""
    ds, D, n = 0.2, 2.5, 30
    g = w.chain_graph(n, ds, param_set=1, params=w.GraphParams(D=D))
    s = orc.Sim(_tet_case())
    s.attach_graph(g)
    W = np.random.default_rng(0).standard_normal(n)
    L = s.graph_laplacian(W)
    assert np.allclose(L[1:-1], D * (W[2:] - 2 * W[1:-1] + W[:-2]) / ds ** 2, rtol=1e-12, atol=1e-10)
    assert np.isclose(L[0], 2 * D * (W[1] - W[0]) / ds ** 2, rtol=1e-12)
    assert np.isclose(L[-1], 2 * D * (W[-2] - W[-1]) / ds ** 2, rtol=1e-12)


def test_tree_laplacian_conserves_and_is_symmetric(orc):
    """Each edge flux leaves one node and enters the other: sum_i vol_i (L W)_i = 0
    with vol_i = half the length of the edges at i; vol_i L_ij is symmetric;
    constants are in the kernel. Branch nodes with several edges included."""
    rng = np.random.default_rng(4)
    n = 40
    xyz, edges = _random_tree(n, rng)
    Dk = rng.uniform(0.5, 3.0, edges.shape[0])
    g = w.Graph(xyz, edges, np.ones(n, np.uint8), np.zeros(n, np.uint8), np.zeros(0, np.int32),
                np.zeros(0, np.int32), np.zeros(0, np.uint8), w.GraphParams(), edge_D=Dk)
    s = orc.Sim(_tet_case())
    s.attach_graph(g)
    length = np.linalg.norm(xyz[edges[:, 0]] - xyz[edges[:, 1]], axis=1)
    vol = np.zeros(n)
    np.add.at(vol, edges[:, 0], 0.5 * length)
    np.add.at(vol, edges[:, 1], 0.5 * length)
    for _ in range(3):
        W = rng.standard_normal(n)
        assert abs(np.dot(vol, s.graph_laplacian(W))) < 1e-11 * np.abs(vol * s.graph_laplacian(W)).sum()
    assert np.abs(s.graph_laplacian(np.full(n, -70.0))).max() < 1e-10
    M = np.stack([s.graph_laplacian(np.eye(n)[k]) for k in range(n)], axis=1)
    A = vol[:, None] * M
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.count_nonzero(np.bincount(edges.ravel(), minlength=n) >= 3) > 3


def test_purkinje_cable_velocity_matches_table2(orc):
    """A Stewart cable with D = m / (chi C_m) (Table 2's Purkinje conductivity)
    conducts at the 4 m/s Table 2 states; the speed converges under refinement."""
    gd = _golden("table2_purkinje.txt")
    D = gd["m_purkinje"] / (gd["chi"] * gd["C_m"])
    cv = []
    for ds, dt in ((0.2, 0.01), (0.1, 0.005), (0.05, 0.0025)):
        n = int(round(20 / ds)) + 1
        g = w.chain_graph(n, ds, param_set=1, stim_nodes=int(round(2.0 / ds)), params=w.GraphParams(D=D))
        s = orc.Sim(_tet_case(dt))
        s.attach_graph(g)
        s.run(int(round(12 / dt)))
        a = s.graph_activation_times()
        x = np.arange(n) * ds
        sel = (x > 5) & (x < 15)
        assert np.all(np.isfinite(a))
        cv.append(np.polyfit(a[sel], x[sel], 1)[0])
    assert abs(cv[-1] - gd["velocity_mm_per_ms"]) < 0.1 * gd["velocity_mm_per_ms"]
    assert cv[0] < cv[1] < cv[2] and (cv[2] - cv[1]) < (cv[1] - cv[0])


def test_resistive_junction_current(orc):
    """The junction current enters each side like an ionic current: with an
    edge-less graph node, one step differs from the uncoupled step by exactly
    -dt g (V_own - V_other) on both sides."""
    dt = 0.02
    gp = w.GraphParams(g_graph=0.7, g_cell=0.09)

    def run(coupled):
        case = _tet_case(dt, amp=0.0)
        s = orc.Sim(case)
        jn = np.array([0], np.int32) if coupled else np.zeros(0, np.int32)
        g = w.Graph(np.array([[0.0, 0.0, 0.0]]), np.zeros((0, 2), np.int32), np.ones(1, np.uint8),
                    np.zeros(1, np.uint8), jn, jn.copy(), np.zeros(jn.size, np.uint8), gp)
        s.attach_graph(g)
        s.graph_set(0, np.array([10.0]))
        s.run(1)
        return s.V[0], s.graph_get(0)[0]

    vm0, vp0 = run(False)
    vm1, vp1 = run(True)
    Vm, Vp = -85.23, 10.0
    assert np.isclose(vm1 - vm0, -dt * gp.g_cell * (Vm - Vp), rtol=1e-10)
    assert np.isclose(vp1 - vp0, -dt * gp.g_graph * (Vp - Vm), rtol=1e-10)


def test_triggered_junction_equals_delayed_stimulus(orc):
    """Sec. 3.3: when the Purkinje node crosses the threshold at t_p, the cells
    within R_S of the junction cell receive the stimulus over
    [t_p + delay, t_p + delay + S_d). The 3D result must equal a run without
    the junction in which those cells get an ordinary stimulus protocol over
    the same whole steps."""
    dt = 0.02
    gp = w.GraphParams(delay_ortho=5.0, amplitude=-80.0, duration=1.0, radius=0.35)

    def build(with_junction):
        case = _tet_case(dt, n_cubes=(12, 4, 2))
        case.threshold = gp.threshold              # graph activation time = junction trigger time
        case.stim_mask[:] = 0
        return case

    case = build(True)
    cen = w.tet_centroids(case.xyz, case.tets)
    jcell = int(np.argmin(np.linalg.norm(cen - cen.mean(0), axis=1)))
    n = 31
    g = w.chain_graph(n, 0.2, start=(0.0, 3.0, 0.0), param_set=1, stim_nodes=10, params=gp)
    g.junction_node = np.array([n - 1], np.int32)
    g.junction_cell = np.array([jcell], np.int32)
    g.junction_mode = np.array([w.JUNC_TRIGGERED], np.uint8)
    s = orc.Sim(case)
    s.attach_graph(g)
    steps = int(round(20 / dt))
    s.run(steps)
    tp = s.graph_activation_times()[-1]
    near = np.linalg.norm(cen - cen[jcell], axis=1) <= gp.radius
    assert np.isfinite(tp) and near.sum() >= 3
    on = [k for k in range(steps) if tp + gp.delay_ortho <= k * dt < tp + gp.delay_ortho + gp.duration]
    assert len(on) == int(round(gp.duration / dt)) and on == list(range(on[0], on[-1] + 1))

    ref_case = build(False)
    ref_case.stim_mask[near] = 2
    ref_case.stimuli = ref_case.stimuli + [w.Stimulus(gp.amplitude, on[0] * dt, len(on) * dt)]
    r = orc.Sim(ref_case)
    r.attach_graph(w.chain_graph(n, 0.2, start=(0.0, 3.0, 0.0), param_set=1, stim_nodes=10, params=gp))
    r.run(steps)
    assert np.allclose(s.V, r.V, rtol=0, atol=1e-9)
    a, b = s.activation_times(), r.activation_times()
    assert np.array_equal(np.isfinite(a), np.isfinite(b)) and np.all(np.isfinite(a[near]))
    assert np.allclose(a[np.isfinite(a)], b[np.isfinite(b)], atol=1e-9)
    assert np.all(a[near] > tp + gp.delay_ortho)


def test_atrial_bundle_velocity_matches_table2(orc):
    """A Courtemanche cable with D = m / (chi C_m) for Table 2's 1D bundle
    conductivity conducts at the 1.54 m/s Table 2 states (within 10 %)."""
    gd = _golden("table2_bundle.txt")
    D = gd["m_bundle"] / (gd["chi"] * gd["C_m"])
    ds, dt, n = 0.2, 0.02, 61
    case = _tet_case(dt)
    case.param_sets = case.param_sets + [w.ParamSet(model=1)]
    g = w.chain_graph(n, ds, param_set=2, stim_nodes=10, params=w.GraphParams(D=D))
    s = orc.Sim(case)
    s.attach_graph(g)
    s.run(int(round(30 / dt)))
    a = s.graph_activation_times()
    x = np.arange(n) * ds
    sel = (x > 3) & (x < 11)
    assert np.all(np.isfinite(a[sel]))
    cv = np.polyfit(a[sel], x[sel], 1)[0]
    assert abs(cv - gd["velocity_mm_per_ms"]) < 0.1 * gd["velocity_mm_per_ms"]


def test_branch_block_by_conductivity(orc):
    """Bundle-branch block (Sec. 5): a segment of a Purkinje cable with its
    conductivity scaled by f. Cable theory gives a speed proportional to
    sqrt(f) inside the segment, so the transit time through it grows by about
    1/sqrt(f) (the segment's ends load it, hence a band); f = 0 (null
    conductivity) blocks conduction completely."""
    ds, dt, n = 0.2, 0.01, 101
    seg = (np.arange(n - 1) >= 40) & (np.arange(n - 1) < 70)      # edges of the 6 mm segment
    transit = {}
    for f in (1.0, 0.25, 0.0):
        g = w.chain_graph(n, ds, param_set=1, stim_nodes=10, params=w.GraphParams(D=2.82))
        g.edge_D = np.where(seg, 2.82 * f, 2.82)
        s = orc.Sim(_tet_case(dt))
        s.attach_graph(g)
        s.run(int(round(25 / dt)))
        a = s.graph_activation_times()
        assert np.all(np.isfinite(a[:41]))
        if f == 0.0:
            assert not np.any(np.isfinite(a[71:]))               # nothing beyond the block
        else:
            assert np.all(np.isfinite(a))
            transit[f] = a[70] - a[40]
    ratio = transit[0.25] / transit[1.0]
    assert 1.6 < ratio < 2.6, ratio
