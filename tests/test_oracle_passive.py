"""Pins of the oracle's tissue step (Sec. 3.2) with a passive membrane
(I_ion = 0, V the only state variable): what is left of the step is forward
Euler on V with the diffusion term of Eq. 7 and the stimulus of Eq. 4, so
V has closed forms.

  - Activation time (Sec. 4: the first upward crossing of a threshold,
    interpolated inside the step). An isolated cell under a constant
    stimulus -A rises by exactly dt A per step, so V is linear in t and the
    crossing time of theta from V0 is (theta - V0) / A. The interpolation
    must return it to rounding; taking t^{n+1} instead of t^n, the wrong end
    of the step, or a downward crossing fails by a sizeable fraction of dt.
  - Pure diffusion conserves sum_c vol_c V_c under zero-flux boundaries,
    step after step, and a stimulus on a set S adds exactly
    dt A sum_{c in S} vol_c per step.
"""
import numpy as np
import pytest

import workloads as w

PASSIVE = 3


def _isolated_cells(v0, dt, amp, theta):
    k = len(v0)
    base = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5]], float)
    xyz = np.concatenate([base + [2.0 * i, 0, 0] for i in range(k)])
    tets = np.arange(4 * k, dtype=np.int32).reshape(k, 4)
    sets = [w.ParamSet(model=PASSIVE)]
    return w.TissueCase("passive cells", xyz, tets, w.fibres_uniform(k), np.zeros(k, np.uint8),
                        np.ones(k, np.uint8), sets, [w.Stimulus(-amp, 0.0, 1000.0)], dt, 0, theta)


def test_passive_model_table(orc):
    assert orc.model_varnames(PASSIVE) == ["V"]


def test_activation_time_closed_form(orc):
    dt, amp, theta = 0.02, 7.25, -20.0
    # starting potentials: crossings at several fractions of a step, one
    # exactly on a step boundary, one cell already above theta (never an
    # upward crossing), a cell starting exactly at theta - dt A
    frac = np.array([0.1, 0.37, 0.5, 0.83, 0.99])
    n_cross = np.array([3, 17, 40, 111, 250])
    t_star = (n_cross + frac) * dt
    v0 = list(theta - amp * t_star) + [theta - amp * 25 * dt, theta + 1.0, theta - amp * dt]
    t_exact = np.concatenate([t_star, [25 * dt, np.inf, dt]])
    case = _isolated_cells(np.array(v0), dt, amp, theta)
    sim = orc.Sim(case)
    sim.set(0, np.array(v0))
    sim.run(300)
    # V is linear in t (no diffusion between isolated cells, no ionic current)
    assert np.allclose(sim.V, np.array(v0) + 300 * dt * amp, rtol=0, atol=1e-11)
    act = sim.activation_times()
    fin = np.isfinite(t_exact)
    assert np.array_equal(np.isfinite(act), fin)
    assert np.abs(act[fin] - t_exact[fin]).max() < 1e-11
    # what the plausible slips would give lies far outside the 1e-11 bound
    t_n1 = np.floor(t_star / dt) * dt + dt * (1 + frac)     # t^{n+1} in place of t^n
    assert np.abs(t_n1 - t_star).min() > 1e-3
    wrong_end = np.floor(t_star / dt) * dt + dt * (1 - frac)  # fraction measured from V^{n+1}
    assert np.abs(wrong_end[frac != 0.5] - t_star[frac != 0.5]).min() > 1e-6


def test_activation_only_upward(orc):
    """A cell driven downward through theta never activates; one that starts
    exactly at theta does not cross from below either."""
    dt, amp, theta = 0.02, -5.0, -20.0
    case = _isolated_cells(np.array([0.0, theta]), dt, amp, theta)
    sim = orc.Sim(case)
    sim.set(0, np.array([0.0, theta]))
    sim.run(200)
    assert np.all(np.isinf(sim.activation_times()))
    assert np.allclose(sim.V, np.array([0.0, theta]) + 200 * dt * amp, atol=1e-11)


@pytest.mark.parametrize("stimulated", [False, True])
def test_pure_diffusion_conservation(orc, stimulated):
    """sum_c vol_c V_c is invariant under pure diffusion with zero-flux
    boundaries (each interior face flux leaves one cell and enters the
    other), and a stimulus -A on a set S adds dt A sum_S vol_c per step."""
    xyz, tets = w.kuhn_box(7, 5, 4, 0.25)
    n = tets.shape[0]
    c = w.tet_centroids(xyz, tets)
    rng = np.random.default_rng(7)
    fib = rng.standard_normal((n, 3))
    fib /= np.linalg.norm(fib, axis=1, keepdims=True)
    mask = ((c[:, 0] < 0.6) & stimulated).astype(np.uint8)
    dt, amp = 0.01, 30.0
    case = w.TissueCase("passive slab", xyz, tets, fib, np.zeros(n, np.uint8), mask,
                        [w.ParamSet(model=PASSIVE)], [w.Stimulus(-amp, 0.0, 2.0)], dt, 0, 1e9)
    sim = orc.Sim(case)
    v0 = rng.uniform(-90.0, 30.0, n)
    sim.set(0, v0)
    vol = orc.Mesh(xyz, tets).cell_info()[1]
    m0 = np.sum(vol * v0)
    n_steps = 400                                  # 200 stimulated steps (2 ms), then 200 more
    sim.run(n_steps)
    m1 = np.sum(vol * sim.V)
    gain = dt * amp * np.sum(vol[mask == 1]) * 200
    assert abs(m1 - (m0 + gain)) < 1e-12 * np.sum(vol * np.abs(v0))
    # the field did diffuse (it is not a trivial invariant of an idle step)
    assert np.abs(sim.V - v0).max() > 1.0
