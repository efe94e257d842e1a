"""Pins of the oracle's second-order Adams-Bashforth option for the
non-gating variables (Sec. 4: the alternative to forward Euler the paper
tries, which lowers the time error although the first-order Rush-Larsen
gates keep the scheme first order overall).

- The first step after a start is forward Euler, bit for bit.
- At the same dt, AB2 has a much smaller error than forward Euler against a
  fine-dt reference, for all three cell models, and both errors fall by
  about 2x when dt halves (first order, bounded by the gates)."""
import numpy as np
import pytest

import workloads as w

T_MS = 400.0


@pytest.mark.parametrize("model", [0, 1, 2])
def test_ab2_first_step_is_forward_euler(orc, model):
    p = w.ParamSet(model=model)
    st = w.Stimulus(-52.0, 0.0, 1.0)
    _, s_fe = orc.cell_run(p, 0.02, 1, st, integrator=0)
    _, s_ab = orc.cell_run(p, 0.02, 1, st, integrator=1)
    assert np.array_equal(s_fe, s_ab)
    _, s_fe = orc.cell_run(p, 0.02, 2, st, integrator=0)
    _, s_ab = orc.cell_run(p, 0.02, 2, st, integrator=1)
    assert not np.array_equal(s_fe, s_ab)                      # the second step differs


@pytest.mark.parametrize("model", [0, 1, 2])
def test_ab2_lowers_time_error(orc, model):
    p = w.ParamSet(model=model)
    st = w.Stimulus(-52.0, 10.0, 1.0)
    fine = 0.0005
    ref, _ = orc.cell_run(p, fine, int(T_MS / fine), st, record_every=int(round(1.0 / fine)), integrator=1)
    err = {}
    for dt in (0.02, 0.01):
        for integ in (0, 1):
            v, _ = orc.cell_run(p, dt, int(round(T_MS / dt)), st, record_every=int(round(1.0 / dt)),
                                integrator=integ)
            err[dt, integ] = np.sqrt(np.mean((v - ref) ** 2))
    for dt in (0.02, 0.01):
        assert err[dt, 1] < 0.6 * err[dt, 0], (dt, err)
    for integ in (0, 1):
        r = err[0.02, integ] / err[0.01, integ]
        assert 1.6 < r < 2.6, (integ, r)
