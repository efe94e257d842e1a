"""Pins of the oracle's 2D Purkinje shell (Sec. 2, Sec. 3.2): triangles in 3D
space with the cell-centred scheme of the myocardium, edges as faces.

- Conservation and row sums, flat and on a curved cylinder patch (the
  shared edge normal makes every edge flux leave one cell and enter the
  other exactly).
- The 2D Kuhn split is centrally symmetric about every interior node: a
  linear field has the exact gradient and no flux divergence, and with D = I
  the operator of x^2/2 is exactly 1 (and of xy exactly 0) in every interior
  cell.
- The cosine mode's decay rate converges under refinement.
- A Stewart shell with Table 2's Purkinje conductivity conducts a planar
  front at the 4 m/s Table 2 states, converging under refinement.
- Shell cells in a simulation with tetrahedra: the two media are separate
  (no face between them), and a conduction-graph junction excites the shell.
"""
import os

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return {k: float(v) for k, v in rows}


def _interior(c, lo, hi, margin):
    return np.all((c[:, :2] > np.asarray(lo) + margin) & (c[:, :2] < np.asarray(hi) - margin), axis=1)


def test_edge_neighbours_and_rejections(orc):
    xyz, tris = w.tri_box(5, 4, 0.5)
    sh = orc.Shell(xyz, tris)
    _, area, nb = sh.cell_info()
    assert np.allclose(area, 0.125)
    n_int_edges = 5 * 4 * 3 - 5 - 4       # edges of the grid minus the boundary ones... per square: 3 edges
    n_edges = (5 + 1) * 4 + 5 * (4 + 1) + 5 * 4
    n_boundary = 2 * (5 + 4)
    assert (nb >= 0).sum() == 2 * (n_edges - n_boundary)
    assert n_int_edges > 0
    for c in range(len(tris)):
        for k in range(3):
            if nb[c, k] >= 0:
                assert c in nb[nb[c, k]]
    with pytest.raises(ValueError):
        orc.Shell(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], float), np.array([[0, 1, 2]]))
    with pytest.raises(ValueError):
        orc.Shell(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], float),
                  np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]]))


@pytest.mark.parametrize("curved", [False, True])
def test_conservation_and_row_sums(orc, curved):
    xyz, tris = w.tri_cylinder(24, 10, 5.0, 6.0) if curved else w.tri_box(12, 9, 0.4)
    sh = orc.Shell(xyz, tris)
    _, area, _ = sh.cell_info()
    rng = np.random.default_rng(2)
    f = rng.standard_normal((len(tris), 3))
    D = np.stack([orc.conductivity(f[k], 2.0, 0.7).ravel() for k in range(len(tris))])
    for _ in range(3):
        out = sh.diffusion(D, rng.standard_normal(len(tris)))
        assert abs(np.sum(out * area)) < 1e-12 * np.sum(np.abs(out * area))
    assert np.abs(sh.diffusion(D, np.full(len(tris), -74.0))).max() < 1e-11


def test_linear_and_quadratic_exact_in_the_interior(orc):
    xyz, tris = w.tri_box(12, 12, 0.5)
    sh = orc.Shell(xyz, tris)
    c, area, _ = sh.cell_info()
    inner = _interior(c, (0, 0), (6, 6), 1.2)
    assert inner.sum() > 60
    I = np.eye(3).ravel()
    a = np.array([0.7, -0.3, 0.0])
    v = c @ a
    g = sh.cell_gradients(sh.node_values(v))
    assert np.abs(g[inner] - a).max() < 1e-12
    assert np.abs(sh.diffusion(I, v)[inner]).max() < 1e-12
    for ax in (0, 1):
        assert np.abs(sh.diffusion(I, 0.5 * c[:, ax] ** 2)[inner] - 1.0).max() < 1e-10
    assert np.abs(sh.diffusion(I, c[:, 0] * c[:, 1])[inner]).max() < 1e-10


def test_cosine_mode_decay_rate_converges(orc):
    errs = []
    for n in (1, 2, 4):
        xyz, tris = w.tri_box(8 * n, 4 * n, 1.0 / n)
        sh = orc.Shell(xyz, tris)
        c, area, _ = sh.cell_info()
        k = np.pi / 8.0
        v = np.cos(k * c[:, 0])
        out = sh.diffusion(2.0 * np.eye(3).ravel(), v)
        lam = -np.sum(out * v * area) / np.sum(v * v * area)
        errs.append(abs(lam / (2.0 * k * k) - 1.0))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.005


def _shell_case(h, dt, length=20.0):
    gd = _golden("table2_purkinje.txt")
    D = gd["m_purkinje"] / (gd["chi"] * gd["C_m"])
    xyz, tris = w.tri_box(int(round(length / h)), 2, h)      # a strip two squares wide
    n = len(tris)
    c = w.tri_centroids(xyz, tris)
    case = w.TissueCase("shell", xyz, np.zeros((0, 4), np.int32), w.fibres_uniform(n), np.zeros(n, np.uint8),
                        (c[:, 0] < 1.0).astype(np.uint8), [w.ParamSet(model=2, D_l=D, D_t=D)],
                        [w.Stimulus(-100.0, 0.0, 1.0)], dt, 0, 0.0, tris=tris)
    return case, c, gd


def test_planar_front_speed_matches_table2(orc):
    """Explicit stability on the shell needs dt rho < 2 with rho ~ 1/h^2
    (about 1400 /ms at h = 0.2 mm), hence the small steps."""
    cv = []
    for h, dt in ((0.4, 0.004), (0.2, 0.001)):
        case, c, gd = _shell_case(h, dt)
        s = orc.Sim(case)
        s.run(int(round(8.0 / dt)))
        a = s.activation_times()
        sel = (c[:, 0] > 5) & (c[:, 0] < 15)
        assert np.all(np.isfinite(a))
        cv.append(np.polyfit(a[sel], c[sel, 0], 1)[0])
    assert abs(cv[-1] - gd["velocity_mm_per_ms"]) < 0.1 * gd["velocity_mm_per_ms"]
    assert cv[0] < cv[1]


def test_shell_with_tets_and_graph_junction(orc):
    """A shell strip beside a tet slab in one simulation: the slab's stimulus
    does not reach the shell (separate media), and a triggered junction from
    a conduction-graph cable excites the shell cells within R_S."""
    xyz_t, tets = w.kuhn_box(8, 4, 2, 0.25)
    xyz_s, tris = w.tri_box(40, 2, 0.2, origin=(0.0, 0.0, 3.0))
    xyz = np.concatenate([xyz_t, xyz_s])
    tris = tris + len(xyz_t)
    nt, ns = len(tets), len(tris)
    ct = w.tet_centroids(xyz_t, tets)
    cs = w.tri_centroids(xyz, tris)
    ps = np.concatenate([np.zeros(nt, np.uint8), np.ones(ns, np.uint8)])
    sm = np.concatenate([(ct[:, 0] < 0.5).astype(np.uint8), np.zeros(ns, np.uint8)])
    case = w.TissueCase("mixed", xyz, tets, w.fibres_uniform(nt + ns), ps, sm,
                        [w.ParamSet(model=0), w.ParamSet(model=2, D_l=2.82, D_t=2.82), w.ParamSet(model=2)],
                        [w.Stimulus(-100.0, 0.0, 1.0)], 0.001, 0, 0.0, tris=tris)
    alone = orc.Sim(case)
    alone.run(3000)
    a = alone.activation_times()
    assert np.isfinite(a[:nt]).any() and not np.isfinite(a[nt:]).any()
    # a cable ending beside the shell's first cells, triggering those within R_S = 0.4 mm
    g = w.chain_graph(20, 0.2, start=(-4.0, 0.2, 3.0), param_set=2, stim_nodes=3,
                      params=w.GraphParams(radius=0.4, amplitude=-300.0, duration=1.0))
    g.junction_node = np.array([19], np.int32)
    g.junction_cell = np.array([nt + int(np.argmin(np.linalg.norm(cs - g.xyz[19], axis=1)))], np.int32)
    g.junction_mode = np.array([w.JUNC_TRIGGERED], np.uint8)
    s = orc.Sim(case)
    s.attach_graph(g)
    s.run(12000)                 # the cable end fires at ~1.5 ms; the stimulus follows 5 ms later
    a = s.activation_times()
    assert np.isfinite(a[nt:]).mean() > 0.9
    assert np.nanmin(a[nt:]) > s.graph_activation_times()[19] + 5.0


def _shell_and_slab(dt, stim_shell=True, stim_slab=False):
    xyz_t, tets = w.kuhn_box(12, 4, 2, 0.25)
    xyz_s, tris = w.tri_box(15, 2, 0.4, origin=(-6.0, 0.0, 0.25))
    xyz = np.concatenate([xyz_t, xyz_s])
    tris = (tris + len(xyz_t)).astype(np.int32)
    nt, ns = len(tets), len(tris)
    ct = w.tet_centroids(xyz_t, tets)
    cs = w.tri_centroids(xyz, tris)
    ps = np.concatenate([np.zeros(nt, np.uint8), np.ones(ns, np.uint8)])
    sm = np.concatenate([((ct[:, 0] > 2.5) if stim_slab else np.zeros(nt, bool)).astype(np.uint8),
                         ((cs[:, 0] < -5.0) if stim_shell else np.zeros(ns, bool)).astype(np.uint8)])
    case = w.TissueCase("shell+slab", xyz, tets, w.fibres_uniform(nt + ns), ps, sm,
                        [w.ParamSet(model=0), w.ParamSet(model=2, D_l=2.82, D_t=2.82)],
                        [w.Stimulus(-100.0, 0.0, 1.0)], dt, 0, 0.0, tris=tris)
    return case, nt, ct, cs


def test_cell_communication_node_equals_delayed_stimulus(orc):
    """Sec. 3.3 between the 2D shell and the 3D myocardium: when the shell's
    source cell crosses the threshold at t_s, the myocardial cells within R_S
    of the target cell receive the stimulus over [t_s + delay, t_s + delay +
    S_d). The result equals a run without the node in which those cells get
    an ordinary stimulus protocol over the same whole steps."""
    dt = 0.004
    gp = w.GraphParams(delay_ortho=5.0, amplitude=-80.0, duration=1.0, radius=0.3)
    case, nt, ct, cs = _shell_and_slab(dt)
    src = nt + int(np.argmin(np.linalg.norm(cs - [-0.3, 0.4, 0.25], axis=1)))    # the shell's far end
    dst = int(np.argmin(np.linalg.norm(ct - [0.2, 0.5, 0.25], axis=1)))
    empty = w.Graph(np.zeros((0, 3)), np.zeros((0, 2), np.int32), np.zeros(0, np.uint8), np.zeros(0, np.uint8),
                    np.array([src], np.int32), np.array([dst], np.int32), np.array([w.JUNC_CELL], np.uint8), gp)
    s = orc.Sim(case)
    s.attach_graph(empty)
    steps = int(round(16 / dt))
    s.run(steps)
    ts = s.activation_times()[src]
    near = np.linalg.norm(ct - ct[dst], axis=1) <= gp.radius
    assert np.isfinite(ts) and near.sum() >= 3
    on = [k for k in range(steps) if ts + gp.delay_ortho <= k * dt < ts + gp.delay_ortho + gp.duration]
    assert len(on) == int(round(gp.duration / dt))
    ref_case, _, _, _ = _shell_and_slab(dt)
    ref_case.stim_mask[:nt][near] = 2
    ref_case.stimuli = ref_case.stimuli + [w.Stimulus(gp.amplitude, on[0] * dt, len(on) * dt)]
    r = orc.Sim(ref_case)
    r.run(steps)
    assert np.allclose(s.V, r.V, rtol=0, atol=1e-9)
    a = s.activation_times()
    assert np.all(a[:nt][near] > ts + gp.delay_ortho) and np.isfinite(a[:nt]).mean() > 0.9


def test_cell_communication_node_two_way(orc):
    """With two-way coupling the myocardium excites the shell back: the
    slab's wave reaches the target cell at t_m, and the source cell is
    stimulated from t_m + delay_anti; without two-way the shell stays at rest."""
    dt = 0.004
    for two_way in (0, 1):
        gp = w.GraphParams(delay_anti=3.0, amplitude=-300.0, duration=1.0, radius=0.3, two_way=two_way)
        case, nt, ct, cs = _shell_and_slab(dt, stim_shell=False, stim_slab=True)
        src = nt + int(np.argmin(np.linalg.norm(cs - [-0.3, 0.4, 0.25], axis=1)))
        dst = int(np.argmin(np.linalg.norm(ct - [0.2, 0.5, 0.25], axis=1)))
        g = w.Graph(np.zeros((0, 3)), np.zeros((0, 2), np.int32), np.zeros(0, np.uint8), np.zeros(0, np.uint8),
                    np.array([src], np.int32), np.array([dst], np.int32), np.array([w.JUNC_CELL], np.uint8), gp)
        s = orc.Sim(case)
        s.attach_graph(g)
        s.run(int(round(14 / dt)))
        a = s.activation_times()
        if two_way:
            assert np.isfinite(a[nt:]).mean() > 0.9 and a[src] > a[dst] + gp.delay_anti
        else:
            assert not np.isfinite(a[nt:]).any()
