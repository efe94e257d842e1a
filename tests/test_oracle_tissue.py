"""Tissue-level pins of the oracle (Sec. 4): the activation front's speed
converges under refinement (increasing toward its limit, as the paper reports
for its benchmark) and follows the anisotropy of the conductivity tensor."""
import numpy as np
import pytest

import workloads as w


def _strip(orc, n, dt, fibre=(1.0, 0.0, 0.0), L=6.0, W=0.5):
    h = 0.5 / n
    xyz, tets = w.kuhn_box(int(round(L / h)), int(round(W / h)), int(round(W / h)), h)
    c = w.tet_centroids(xyz, tets)
    N = tets.shape[0]
    case = w.TissueCase("strip", xyz, tets, w.fibres_uniform(N, fibre), np.zeros(N, np.uint8),
                        (c[:, 0] < 1.0).astype(np.uint8), [w.ParamSet()],
                        [w.Stimulus(-52.0, 0.0, 1.0)], dt, int(round(24 / dt)), -20.0)
    s = orc.Sim(case)
    s.run(case.n_steps)
    a = s.activation_times()
    s0, s1 = np.abs(c[:, 0] - 2.0) < h, np.abs(c[:, 0] - 5.0) < h
    return 3.0 / (a[s1].mean() - a[s0].mean())


def test_conduction_velocity_converges_under_refinement(orc):
    cv = [_strip(orc, n, dt) for n, dt in ((1, 0.02), (2, 0.01), (4, 0.005))]
    assert cv[0] < cv[1] < cv[2]
    d1, d2 = cv[1] - cv[0], cv[2] - cv[1]
    assert d2 < 0.75 * d1
    assert 0.5 < cv[2] < 1.0   # mm/ms, ventricular range for D_l = 0.154 mm^2/ms


def test_conduction_velocity_anisotropy(orc):
    """CV scales like sqrt(D): along vs across the fibre the ratio approaches
    sqrt(D_l / D_t) = 2."""
    cl = _strip(orc, 2, 0.01, (1.0, 0.0, 0.0))
    ct = _strip(orc, 2, 0.01, (0.0, 1.0, 0.0))
    assert 1.7 < cl / ct < 2.3


def test_slab_activation_map(orc):
    """16x16x4-cube slab, stimulus x < 1 mm: every cell activates once within
    20 ms, later further from the stimulus, inside the step it crossed in."""
    case = w.slab_case()
    s = orc.Sim(case)
    s.run(1000)
    a = s.activation_times()
    c = w.tet_centroids(case.xyz, case.tets)
    assert np.all(np.isfinite(a)) and a.min() >= 0.0 and a.max() < 20.0
    far, near = a[c[:, 0] > 7.0].mean(), a[c[:, 0] < 1.0].mean()
    assert far > near + 5.0
    order = np.argsort(c[:, 0])
    xs = c[order, 0]
    bins = [a[order][(xs >= k) & (xs < k + 1)].mean() for k in range(8)]
    assert all(b2 > b1 for b1, b2 in zip(bins[1:], bins[2:]))
    assert s.step_index == 1000


def test_tissue_charge_balance(orc):
    """Zero-flux boundaries and face fluxes that leave one cell and enter its
    neighbour make the diffusion term sum to zero over the cells (weighted
    by volume), and TP06 moves in ions exactly the charge its V equation
    moves (stimulus carried by K+). So the volume-weighted charge balance of
    the slab, C_m V - F [V_c (Na_i + K_i) + 2 sum volume x total calcium],
    stays constant to rounding while the front crosses it. A diffusion term
    divided by the wrong volume, or a boundary face that lets current out,
    breaks it by the order of the C_m V swing."""
    from test_oracle_cells import _charge
    case = w.slab_case()
    x = case.xyz[case.tets]
    vol = np.abs(np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])) / 6.0
    s = orc.Sim(case)
    names = orc.model_varnames(0)

    def balance():
        state = np.stack([s.V if n == "V" else s.get(k) for k, n in enumerate(names)])
        q = _charge(orc, 0, state)
        return float(np.dot(vol, q)), float(np.dot(vol, state[0]))
    q0, v0 = balance()
    for n in (100, 500, 1000):
        s.run(n - s.step_index)
        q, v = balance()
        swing = 0.185 * abs(v - v0)
        assert swing > 100.0 and abs(q - q0) < 1e-9 * swing
