"""Physiological pins of the oracle's cell models (Sec. 3.1, Sec. 5) and of
the Rush-Larsen / forward-Euler scheme (Sec. 3.2).

Parity with the published model traces is unpinned (the model papers' figures
and code are not available); these tests pin what the method paper and the
models' physiology fix: resting potentials, action-potential duration and
plateau, automaticity, and the time-integration properties."""
import numpy as np
import pytest

import workloads as w

DT = 0.02


def _apd(v, dt, frac):
    rest, peak = v[0], v.max()
    ip = int(v.argmax())
    up = int(np.argmax(v > 0.5 * (rest + peak)))
    thr = peak - frac * (peak - rest)
    i = ip
    while i < len(v) and v[i] > thr:
        i += 1
    return (i - up) * dt


def _paced(orc, ps, amp, dur, beats=6, bcl=1000.0, dt=DT):
    stim = orc.Stim(amp, 0.0, dur, bcl)
    n_beat = int(round(bcl / dt))
    v, st = orc.cell_run(ps, dt, n_beat * beats, stim, 1)
    return v[-n_beat - 1:], st


@pytest.fixture(scope="module")
def tp06_beats(orc):
    return {var: _paced(orc, w.ParamSet(model=0, variant=var), -52.0, 1.0)
            for var in (0, 1, 2)}


def test_tp06_rest_and_peak(tp06_beats):
    """TP06 rests near -85 mV (Sec. 5) with an overshooting upstroke."""
    for var, (v, _) in tp06_beats.items():
        assert -87.0 <= v[0] <= -84.0
        assert 25.0 <= v.max() <= 50.0


def test_tp06_apd_and_variant_order(tp06_beats):
    """Plateau of about 300 ms (Sec. 5); the M cell has the longest APD; the
    epi cell has a deeper early-repolarisation notch than the endo cell."""
    apd = {k: _apd(v, DT, 0.9) for k, (v, _) in tp06_beats.items()}
    assert 260.0 <= apd[0] <= 340.0
    assert apd[1] > apd[0] + 40.0 and apd[1] > apd[2] + 40.0
    assert abs(apd[2] - apd[0]) < 20.0
    notch = {}
    for k in (0, 2):
        v = tp06_beats[k][0]
        ip = int(v.argmax())
        notch[k] = v[ip:ip + int(30 / DT)].min()
    assert notch[0] < notch[2] - 5.0


def test_tp06_unstimulated_stays_at_rest(orc):
    v, _ = orc.cell_run(w.ParamSet(model=0), DT, 50000, None, 100)
    assert np.all((v > -87.0) & (v < -84.0))


def test_courtemanche_rest_and_repolarisation(orc):
    """Courtemanche rests near -80 mV and repolarises within a few hundred ms
    (Sec. 5)."""
    v, _ = _paced(orc, w.ParamSet(model=1), -20.0, 2.0)
    assert -82.0 <= v[0] <= -79.0
    assert v.max() > 10.0
    assert 120.0 <= _apd(v, DT, 0.5) <= 260.0
    assert _apd(v, DT, 0.9) <= 360.0


def test_stewart_high_peak_plateau_and_automaticity(orc):
    """Stewart Purkinje cell: high depolarisation peak and a plateau of about
    250 ms (Sec. 5); unstimulated, I_f makes it fire on its own."""
    v, _ = _paced(orc, w.ParamSet(model=2), -52.0, 1.0)
    assert v.max() > 40.0
    assert 150.0 <= _apd(v, DT, 0.5) <= 320.0
    v, _ = orc.cell_run(w.ParamSet(model=2), DT, 150000, None, 1)
    up = np.flatnonzero((v[:-1] < 0.0) & (v[1:] >= 0.0))
    assert len(up) >= 1


@pytest.mark.parametrize("model", [0, 1, 2])
def test_rush_larsen_exact_for_frozen_voltage(orc, model):
    """With V frozen, the RL update of a gate is its exact exponential
    solution, so 1 step of 4*dt equals 4 steps of dt for every gate whose
    rates depend on V only (the FE variables do not have this property)."""
    ps = w.ParamSet(model=model)
    names = orc.model_varnames(model)
    gates = {0: ["m", "h", "j", "xr1", "xr2", "xs", "r", "s", "d", "f", "f2"],
             1: ["m", "h", "j", "oa", "oi", "ua", "ui", "xr", "xs", "d", "f"],
             2: ["m", "h", "j", "xr1", "xr2", "xs", "r", "s", "d", "f", "f2", "y"]}[model]
    s0 = orc.model_init(ps)
    s0[0] = -20.0
    a = s0.copy()
    for _ in range(4):
        orc.model_step(a, 0.01, 0.0, ps)
    b = s0.copy()
    orc.model_step(b, 0.04, 0.0, ps)
    for g in gates:
        k = names.index(g)
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-15), g


def test_first_order_in_time(orc):
    """FE/RL is first order in dt (Sec. 4): the error of V at a fixed time
    halves when dt halves."""
    ps = w.ParamSet(model=0)
    T = 30.0

    def v_at(dt):
        n = int(round(T / dt))
        v, _ = orc.cell_run(ps, dt, n, orc.Stim(-52.0, 0.0, 1.0, 0.0), n)
        return v[-1]

    ref = v_at(0.000625)
    e = [abs(v_at(dt) - ref) for dt in (0.02, 0.01, 0.005)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 1.6 < r1 < 2.6 and 1.6 < r2 < 2.6


def test_stimulus_schedule(orc):
    """Eq. 4 with whole steps: on for round(S_d/dt) steps from the onset,
    repeating every round(period/dt) steps."""
    s = orc.Stim(-52.0, 0.0, 1.0, 0.0)
    on = [orc.stim_active(s, 0.02, n) for n in range(60)]
    assert on == [True] * 50 + [False] * 10
    s = orc.Stim(-52.0, 2.0, 0.5, 10.0)
    on = [orc.stim_active(s, 0.5, n) for n in range(30)]
    assert [n for n in range(30) if on[n]] == [4, 24]


# TP06 / Stewart geometry and calcium buffers (the models' parameter tables)
_F, _CM, _VC, _VSR, _VSS = 96485.3415, 0.185, 0.016404, 0.001094, 0.00005468
_BUF = {"Ca_i": (0.2, 0.001, _VC), "Ca_SR": (10.0, 0.3, _VSR), "Ca_SS": (0.4, 0.00025, _VSS)}


def _charge(orc, model, s):
    """C_m V minus the ionic charge held in the cell, F [V_c (Na_i + K_i) +
    2 sum over compartments of volume x total (free + buffered) calcium]. The
    model's V equation, C_m dV/dt = -C_m (I_ion + I_stim), and its
    concentration equations move the same charge (the stimulus is carried by
    K+), so this is constant along any trajectory."""
    names = orc.model_varnames(model)
    x = {n: s[k] for k, n in enumerate(names)}
    ca = sum(vol * (x[n] + B * x[n] / (x[n] + K)) for n, (B, K, vol) in _BUF.items())
    return _CM * x["V"] - _F * (_VC * (x["Na_i"] + x["K_i"]) + 2.0 * ca)


@pytest.mark.parametrize("model,variant", [(0, 0), (0, 1), (0, 2), (2, 0)])
@pytest.mark.parametrize("integrator", [0, 1])
def test_charge_conservation(orc, model, variant, integrator):
    """Forward Euler (or AB2) on the currents and on the buffered calcium
    totals, Rush-Larsen on the gates: every current appears in the V equation
    and in the concentration equations with the same sign and valence, the
    SR and subspace fluxes only move calcium between compartments, so the
    charge balance holds step by step to rounding -- through the stimulus,
    the upstroke and the whole action potential. A dropped current, a wrong
    valence or a wrong compartment volume breaks it by about C_m x (the
    current) x (the time it flows), orders of magnitude above the bound."""
    ps = w.ParamSet(model=model, variant=variant)
    s = orc.model_init(ps)
    q0 = _charge(orc, model, s)
    stim = orc.Stim(-52.0, 0.0, 1.0, 0.0)
    v, s = orc.cell_run(ps, DT, 200, stim, 1, s, integrator=integrator)       # stimulus and upstroke
    q1 = _charge(orc, model, s)
    v2, s = orc.cell_run(ps, DT, 20000, None, 100, s, integrator=integrator)  # the rest of a 400 ms beat
    q2 = _charge(orc, model, s)
    swing = _CM * (max(v.max(), v2.max()) - min(v.min(), v2.min()))
    assert swing > 15.0                          # an action potential happened
    assert abs(q1 - q0) < 1e-6 * swing and abs(q2 - q0) < 1e-6 * swing



# Courtemanche geometry and calcium buffers (the model's parameter table)
_CRN = dict(F=96.4867, Cm=100.0, Vi=13668.0, Vup=1109.52, Vrel=96.48)


def _charge_crn(orc, s):
    """The same balance for Courtemanche: cytosolic calcium buffered by
    calmodulin and troponin, release-store calcium by calsequestrin, the
    uptake store unbuffered."""
    x = dict(zip(orc.model_varnames(1), s))
    cai, cr = x["Ca_i"], x["Ca_rel"]
    cat = cai + 0.05 * cai / (cai + 0.00238) + 0.07 * cai / (cai + 0.0005)
    crt = cr + 10.0 * cr / (cr + 0.8)
    c = _CRN
    return c["Cm"] * x["V"] - c["F"] * (c["Vi"] * (x["Na_i"] + x["K_i"])
                                        + 2.0 * (c["Vi"] * cat + c["Vup"] * x["Ca_up"] + c["Vrel"] * crt))


def test_courtemanche_charge_balance_first_order():
    """Courtemanche carries its stimulus on no ion, so the balance moves by
    exactly the stimulus charge, C_m x 52 x 1 ms; and it advances the free
    cytosolic and release-store calcium with the buffering factor, so what
    remains is a first-order error: it halves with dt and extrapolates to
    zero. A dropped or mis-signed current would leave a part that does not
    shrink with dt."""
    import oracle as orc
    ps = w.ParamSet(model=1)
    res, swing = {}, 0.0
    for dt in (0.02, 0.01, 0.005):
        s = orc.model_init(ps)
        q0 = _charge_crn(orc, s)
        v, s = orc.cell_run(ps, dt, int(round(400.0 / dt)), orc.Stim(-52.0, 0.0, 1.0, 0.0), 1, s)
        res[dt] = _charge_crn(orc, s) - q0 - _CRN["Cm"] * 52.0 * int(round(1.0 / dt)) * dt
        swing = _CRN["Cm"] * (v.max() - v.min())
    assert swing > 5000.0
    for a, b in ((0.02, 0.01), (0.01, 0.005)):
        assert abs(res[a] / res[b] - 2.0) < 0.05
        assert abs(2.0 * res[b] - res[a]) < 1e-3 * swing
