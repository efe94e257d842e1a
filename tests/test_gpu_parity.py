"""Parity of the CUDA path with the FP64 oracle on the same seeded inputs,
through the C ABI (ep_mesh_create / ep_params_set / ep_step / ep_read_state
/ ep_activation_times)."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, isolated_cells, run_gpu, run_oracle, tolerances

pytestmark = pytest.mark.gpu

PRECISIONS = ["mixed", "plain"]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2112_12854_b300 import ep
    c = ep.Context()
    yield c
    c.close()


def _prec(name):
    from paper_2112_12854_b300 import ep
    return ep.EP_FP32_MIXED if name == "mixed" else ep.EP_FP64_PLAIN


@pytest.mark.parametrize("pname", PRECISIONS)
def test_single_cells_all_models(ctx, pname):
    """Each cell model (TP06 epi/M/endo, Courtemanche, Stewart) as isolated
    cells paced at 2 Hz for 600 ms: V and every state variable against the
    oracle."""
    import oracle
    from paper_2112_12854_b300 import ep
    prec = _prec(pname)
    tv, _ = tolerances(prec)
    mv = [(0, 0), (0, 1), (0, 2), (1, 0), (2, 0)]
    case = isolated_cells(mv)
    outs = [2500, 10000, 30000]
    ref, _, osim = run_oracle(case, outs)
    got, _, job = run_gpu(ctx, case, outs, prec)
    for n in outs:
        err = np.abs(got[n] - ref[n]).max()
        assert err <= tv, (n, err)
    for k, (m, _) in enumerate(mv):
        names = oracle.model_varnames(m)
        for var in range(1, len(names)):
            g = job.read(var, model=m)[k]
            r = osim.get(var)[k]
            tol = 1e-9 if pname == "plain" else 2e-3
            assert abs(g - r) <= tol * max(abs(r), 1e-3), (names[var], g, r)
    job.destroy()


@pytest.mark.parametrize("pname", PRECISIONS)
def test_slab_6144_cells_1000_steps(ctx, pname):
    """The 16x16x4-cube TP06 slab (6144 cells), 1000 steps of 0.02 ms: V at
    steps 250/500/1000 and the activation map (threshold -20 mV)."""
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    case = w.slab_case()
    outs = [250, 500, 1000]
    ref, ract, sim = run_oracle(case, outs)
    got, gact, job = run_gpu(ctx, case, outs, prec)
    for n in outs:
        d = np.abs(got[n] - ref[n])
        print(pname, "step", n, "|dV| max", d.max(), "mean", d.mean(), "p99", np.percentile(d, 99))
        assert d.max() <= tv
    e = act_error(gact, ract)
    print(pname, "max|dt_act|", e)
    assert np.all(np.isfinite(ract)) and e <= ta
    # every state variable at step 1000, relative to its largest magnitude on the slab
    # (gates in [0, 1], concentrations in mM): 1e-3 for FP32 mixed, 1e-9 for FP64 plain
    from paper_2112_12854_b300 import ep
    rel_tol = 1e-9 if prec == ep.EP_FP64_PLAIN else 1e-3
    for v, name in enumerate(ep.model_varnames(ep.EP_TP06)):
        if v == 0:
            continue
        r, g = sim.get(v), job.read(v)
        rel = np.abs(g - r).max() / np.abs(r).max()
        print(pname, f"{name:>6s} max|d|/max|ref| {rel:.2e}")
        assert rel <= rel_tol, name
    job.destroy()


@pytest.mark.parametrize("pname", PRECISIONS)
def test_mixed_models_ragged_slab(ctx, pname):
    """A ragged slab (13x7x3 cubes, 1638 cells: several tiles and a ragged
    tail) split into TP06 / Courtemanche / Stewart thirds along x, fibres
    rotating with depth, two stimuli."""
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    xyz, tets = w.kuhn_box(13, 7, 3, 0.25)
    c = w.tet_centroids(xyz, tets)
    n = tets.shape[0]
    model = np.where(c[:, 0] < 1.1, 0, np.where(c[:, 0] < 2.2, 1, 2))
    sets = [w.ParamSet(model=0, variant=2), w.ParamSet(model=1), w.ParamSet(model=2)]
    stim = ((c[:, 0] < 0.5).astype(np.uint8) | ((c[:, 0] > 2.9).astype(np.uint8) << 1))
    case = w.TissueCase("mix", xyz, tets, w.fibres_transmural(c[:, 2], 0.0, 0.75), model.astype(np.uint8),
                        stim, sets, [w.Stimulus(-52.0, 0.0, 1.0), w.Stimulus(-40.0, 5.0, 2.0)],
                        0.01, 0, -10.0)
    outs = [300, 1000, 2500]
    ref, ract, _ = run_oracle(case, outs)
    got, gact, job = run_gpu(ctx, case, outs, prec)
    for k in outs:
        assert np.abs(got[k] - ref[k]).max() <= tv
    assert act_error(gact, ract) <= ta
    job.destroy()


def test_batched_equals_alone_bitwise(ctx):
    """A job gives bit-identical results alone and batched with others
    (per-cell gathers, no atomics), through the captured-graph path."""
    from paper_2112_12854_b300 import ep
    a_case = w.slab_case(nx=9, ny=5, nz=3, h=0.5)
    b_case = w.slab_case(nx=17, ny=6, nz=2, h=0.25, D_l=0.1, D_t=0.05)
    alone = ep.job_from_case(ctx, a_case)
    alone.step(150)
    va, aa = alone.V, alone.activation_times()
    ja, jb = ep.job_from_case(ctx, a_case), ep.job_from_case(ctx, b_case)
    jc = ep.job_from_case(ctx, b_case, precision=ep.EP_FP64_PLAIN)
    ep.step([jb, ja, jc], 150)
    assert np.array_equal(ja.V, va)
    assert np.array_equal(ja.activation_times(), aa)
    assert ja.step_index == jb.step_index == jc.step_index == 150
    for j in (alone, ja, jb, jc):
        j.destroy()


def test_graph_replay_equals_single_steps(ctx):
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=8, ny=8, nz=2)
    j1, j2 = ep.job_from_case(ctx, case), ep.job_from_case(ctx, case)
    j1.step(200)            # graph of 32 steps x 6 + 8 direct
    for _ in range(200):
        j2.step(1)
    assert np.array_equal(j1.V, j2.V)
    for m in range(1, 19):
        assert np.array_equal(j1.read(m), j2.read(m))
    j1.destroy()
    j2.destroy()


def test_checkpoint_resume_exact(ctx):
    """ep_read_state / ep_write_state / ep_set_step_index restore a job
    exactly: the resumed run equals the uninterrupted one bit for bit."""
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=10, ny=6, nz=2)
    ref = ep.job_from_case(ctx, case)
    ref.step(137)
    snap = {v: ref.read(v) for v in range(19)}
    act = ref.activation_times()
    ref.step(163)
    new = ep.job_from_case(ctx, case)
    for v, vals in snap.items():
        new.write(v, vals)
    new.step_index = 137
    new.step(163)
    assert new.step_index == 300
    assert np.array_equal(new.V, ref.V)
    for v in range(1, 19):
        assert np.array_equal(new.read(v), ref.read(v))
    # activation recorded before the snapshot is not in the state: compare after it
    fin = np.isfinite(act)
    ga = new.activation_times()
    assert np.array_equal(ga[~fin], ref.activation_times()[~fin])
    ref.destroy()
    new.destroy()


def test_fp32_state_transfers_exact(ctx):
    """ep_read_state_f32 / ep_write_state_f32 / ep_activation_times_f32 move
    the variables an FP32 job stores in FP32 exactly: each read equals the
    FP64 read rounded to FP32 (the stored value), and a checkpoint taken with
    them (the compensated concentrations through the FP64 calls) resumes bit
    for bit, over three cell models. The compensated variables and FP64 jobs
    are refused with EP_EINVAL."""
    from paper_2112_12854_b300 import ep
    xyz, tets = w.kuhn_box(12, 6, 3, 0.25)
    c = w.tet_centroids(xyz, tets)
    ps = np.where(c[:, 0] < 1.0, 0, np.where(c[:, 0] < 2.0, 1, 2)).astype(np.uint8)
    case = w.TissueCase("mix3", xyz, tets, w.fibres_uniform(len(tets)), ps, (c[:, 0] < 0.6).astype(np.uint8),
                        [w.ParamSet(model=0), w.ParamSet(model=1), w.ParamSet(model=2)],
                        [w.Stimulus(-60.0, 0.0, 1.0)], 0.02, 0, -20.0)
    ref = ep.job_from_case(ctx, case)
    ref.step(140)
    snap = {}
    for m in range(3):
        comp = ep.model_var_compensated(m)
        assert any(comp) and not comp[0]
        for v in range(len(comp)):
            d = ref.read(v, model=m)
            if comp[v]:
                with pytest.raises(ep.EPError) as e:
                    ref.read_f32(v, model=m)
                assert e.value.code == ep.EP_EINVAL
                snap[m, v] = d
            else:
                f = ref.read_f32(v, model=m)
                assert np.array_equal(f, d.astype(np.float32), equal_nan=True), (m, v)
                snap[m, v] = f
    a32 = ref.activation_times_f32()
    assert np.array_equal(a32, ref.activation_times().astype(np.float32))
    assert np.isfinite(a32).any()
    ref.step(160)
    new = ep.job_from_case(ctx, case)
    for (m, v), vals in snap.items():
        if vals.dtype == np.float32:
            new.write_f32(v, vals, model=m)
        else:
            new.write(v, vals, model=m)
    new.step_index = 140
    new.step(160)
    for m in range(3):
        for v in range(len(ep.model_varnames(m))):
            assert np.array_equal(new.read(v, model=m), ref.read(v, model=m), equal_nan=True), (m, v)
    plain = ep.job_from_case(ctx, case, precision=ep.EP_FP64_PLAIN)
    for call in (lambda: plain.read_f32(0), lambda: plain.write_f32(0, np.zeros(plain.n_cells, np.float32)),
                 lambda: plain.activation_times_f32()):
        with pytest.raises(ep.EPError) as e:
            call()
        assert e.value.code == ep.EP_EINVAL
    for j in (ref, new, plain):
        j.destroy()


def test_errors_reported(ctx):
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=4, ny=4, nz=2, h=0.25)
    j = ctx.mesh(case.xyz, case.tets, param_set=case.param_set, fibre=case.fibre)
    with pytest.raises(ep.EPError) as e:
        j.step(1)
    assert e.value.code == ep.EP_ESTATE
    with pytest.raises(ep.EPError) as e:
        j.set_params(ep.make_params(0.2, case.param_sets, case.stimuli))
    assert e.value.code == ep.EP_EUNSTABLE
    j.set_params(ep.make_params(0.01, case.param_sets, case.stimuli))
    with pytest.raises(ep.EPError) as e:
        ep.step([j, j], 1)
    assert e.value.code == ep.EP_EINVAL
    assert j.check_finite()
    v = j.V
    v[3] = np.nan
    j.write(0, v)
    assert not j.check_finite()
    j.destroy()
