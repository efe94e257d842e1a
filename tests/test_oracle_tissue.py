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
