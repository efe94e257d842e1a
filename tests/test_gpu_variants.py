"""The cell kernel's launch-shape variants (ep_autotune / ep_set_cell_variant)
change only the launch configuration: every variant must give bitwise the
same state, and the autotuner's steps are ordinary time steps."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_all_cell_variants_bitwise_identical(pname):
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    case = w.slab_case(nx=11, ny=7, nz=3, h=0.5)
    ctx = ep.Context()
    ref = None
    for v in range(ep.N_CELL_VARIANTS):
        ep.set_cell_variant(ctx, prec, v)
        j = ep.job_from_case(ctx, case, precision=prec)
        j.step(120)
        state = [j.read(k) for k in range(19)] + [j.activation_times()]
        if ref is None:
            ref = state
        else:
            for a, b in zip(state, ref):
                assert np.array_equal(a, b, equal_nan=True), v
        j.destroy()
    ctx.close()


def test_autotune_steps_are_real_steps():
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=9, ny=6, nz=3, h=0.5)
    ctx = ep.Context()
    a = ep.job_from_case(ctx, case)
    chosen, ms = ep.autotune([a], 4)
    assert 0 <= chosen[0] < ep.N_CELL_VARIANTS and chosen[1] == -1
    assert np.all(ms[0] > 0)
    assert a.step_index == 4 * ep.N_CELL_VARIANTS
    a.step(50)
    b = ep.job_from_case(ctx, case)
    b.step(4 * ep.N_CELL_VARIANTS + 50)
    assert np.array_equal(a.V, b.V)
    ctx.close()


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_variants_bitwise_on_mixed_models_and_graph(pname):
    """All launch variants, including the staged kernel (bulk-copied tiles,
    with its fallbacks for region starts and ragged tails that are not
    16-byte aligned), on TP06 / Courtemanche / Stewart regions of uneven size
    with a conduction graph and junction cells. The full staged kernel and
    the 128-register shapes agree bitwise; under the tighter register limits
    of the 80- and 96-register shapes the compiled Courtemanche arithmetic
    can round differently in the last bits, so those are held to 1e-4 mV."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    xyz, tets = w.kuhn_box(10, 7, 3, 0.25)
    n = tets.shape[0]
    c = w.tet_centroids(xyz, tets)
    ps = np.where(np.arange(n) < 421, 0, np.where(np.arange(n) < 899, 1, 2)).astype(np.uint8)
    case = w.TissueCase("slab", xyz, tets, w.fibres_uniform(n), ps, (c[:, 0] < 0.6).astype(np.uint8),
                        [w.ParamSet(model=0), w.ParamSet(model=1), w.ParamSet(model=2)],
                        [w.Stimulus(-80.0, 0.0, 1.0)], 0.02, 0, -20.0)
    g = w.chain_graph(30, 0.2, start=(0.0, 1.0, 0.4), param_set=2, stim_nodes=0)
    g.junction_node = np.array([29], np.int32)
    g.junction_cell = np.array([int(np.argmin(np.linalg.norm(c - g.xyz[29], axis=1)))], np.int32)
    g.junction_mode = np.array([w.JUNC_RESISTIVE], np.uint8)
    g.params = w.GraphParams(g_cell=4.0)
    ctx = ep.Context()
    ref = None
    for v in range(ep.N_CELL_VARIANTS):
        ep.set_cell_variant(ctx, prec, v)
        # 32-bit indices: the staged variants (6, 7) run only on those
        j = ep.job_from_case(ctx, case, precision=prec, index_width=32)
        j.attach_graph(g, node_model=np.full(30, 2, np.uint8))
        j.step(150)
        state = [j.read(k, model=m) for m in range(3) for k in range(len(ep.model_varnames(m)))]
        state += [j.activation_times(), j.graph_read(0, model=2)]
        if ref is None:
            ref = state
        else:
            for a, b in zip(state, ref):
                if v in (2, 6):
                    assert np.array_equal(a, b, equal_nan=True), v
                else:
                    assert np.allclose(a, b, rtol=1e-5, atol=1e-4, equal_nan=True), v
        assert j.check_finite()
        j.destroy()
    ctx.close()


def _three_model_case():
    xyz, tets = w.kuhn_box(13, 7, 3, 0.25)
    c = w.tet_centroids(xyz, tets)
    model = np.where(c[:, 0] < 1.1, 0, np.where(c[:, 0] < 2.2, 1, 2)).astype(np.uint8)
    sets = [w.ParamSet(model=0, variant=2), w.ParamSet(model=1), w.ParamSet(model=2)]
    stim = ((c[:, 0] < 0.5).astype(np.uint8) | ((c[:, 0] > 2.9).astype(np.uint8) << 1))
    return w.TissueCase("mix", xyz, tets, w.fibres_transmural(c[:, 2], 0.0, 0.75), model, stim, sets,
                        [w.Stimulus(-52.0, 0.0, 1.0), w.Stimulus(-40.0, 5.0, 2.0)], 0.01, 0, -10.0)


def _state(j):
    from paper_2112_12854_b300 import ep
    st = [j.read(k, model=m) for m in range(3) for k in range(len(ep.model_varnames(m)))]
    return st + [j.activation_times()]


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_index_widths_bitwise_identical(pname):
    """The gather indices stored as 16-bit offsets (cell gathers and node
    table: index_width 16), as the default mix (16-bit cell gathers, 32-bit
    node table) and as 32-bit indices (index_width 32) give bitwise the same
    state, each alone and batched together -- a batch of mixed node-table
    forms takes the node kernel that reads both (TP06 / Courtemanche /
    Stewart regions, two stimuli, 1638 cells: several tiles, ragged
    tails)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    case = _three_model_case()
    ctx = ep.Context()
    a16 = ep.job_from_case(ctx, case, precision=prec, index_width=16)
    a32 = ep.job_from_case(ctx, case, precision=prec, index_width=32)
    b16 = ep.job_from_case(ctx, case, precision=prec, index_width=16)
    b32 = ep.job_from_case(ctx, case, precision=prec)                 # the default: 16-bit cells only
    assert a16.info()["index_width"] == 16 and a32.info()["index_width"] == 32
    assert a16.info()["node_index_width"] == 16 and a32.info()["node_index_width"] == 32
    assert (b32.info()["index_width"], b32.info()["node_index_width"]) == (16, 32)
    assert a16.info()["device_bytes"] < a32.info()["device_bytes"]
    a16.step(300)
    a32.step(300)
    ep.step([b16, b32], 300)
    ref = _state(a32)
    for j in (a16, b16, b32):
        for x, y in zip(_state(j), ref):
            assert np.array_equal(x, y, equal_nan=True)
    assert np.isfinite(ref[-1]).any()
    ctx.close()


def test_index_widths_bitwise_identical_bidomain():
    """The bidomain solve (node passes and fluxes of the elliptic operator)
    reads the same 16-bit or 32-bit indices: V and v_e agree bitwise."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    case = w.slab_case(nx=12, ny=8, nz=3, h=0.25)
    ctx = ep.Context()
    jobs = [ep.job_from_case(ctx, case, index_width=iw) for iw in (16, 32)]
    for j in jobs:
        j.enable_bidomain(0.62 / 1.4, 0.24 / 1.4)
        j.step(80)
    assert np.array_equal(jobs[0].V, jobs[1].V)
    assert np.array_equal(jobs[0].ve, jobs[1].ve)
    ctx.close()


@pytest.mark.parametrize("pname", ["mixed", "plain"])
@pytest.mark.parametrize("fused,plain", [(8, 4), (9, 1)])
def test_fused_step_equals_two_launch_step(pname, fused, plain):
    """The fused step (node values and cell update in one launch, node tiles
    and cell tiles in dependency order) gives bitwise the state of the
    two-launch step with the same block shape and register budget (128 x 6
    and 256 x 3), on a slab large enough for many tiles of both kinds to be
    in flight at once (27648 cells, 108 cell tiles, 22 node tiles)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    prec = ep.EP_FP32_MIXED if pname == "mixed" else ep.EP_FP64_PLAIN
    case = w.slab_case(nx=24, ny=24, nz=8, h=0.25, stim_x=0.6)
    ctx = ep.Context()
    out = []
    for v in (plain, fused):
        ep.set_cell_variant(ctx, prec, v)
        j = ep.job_from_case(ctx, case, precision=prec)
        j.step(400)                                          # captured-graph replay and direct launches
        out.append([j.read(k) for k in range(19)] + [j.activation_times()])
        assert j.check_finite()
        j.destroy()
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)
    assert np.isfinite(out[0][-1]).sum() > 1000
    ctx.close()


@pytest.mark.parametrize("variant", [8, 9])
def test_fused_step_batched_equals_alone(variant):
    """One fused launch serves a batch of jobs of different sizes and index
    forms (work lists concatenated, a ready flag per node tile and a launch
    counter per job): every job is bitwise what it is stepped alone, with
    forward Euler and AB2 FP32 jobs and a bidomain job in the FP32 batch, and
    an FP64 job in its own group."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    ctx = ep.Context()
    for p in (ep.EP_FP32_MIXED, ep.EP_FP64_PLAIN):
        ep.set_cell_variant(ctx, p, variant)
    specs = [(w.slab_case(nx=9, ny=5, nz=3, h=0.5), {}, None),
             (w.slab_case(nx=20, ny=14, nz=4, h=0.25, D_l=0.1, D_t=0.05), {"index_width": 32}, None),
             (w.slab_case(nx=8, ny=6, nz=3, h=0.5), {"integrator": 1}, None),     # AB2: dt rho < 1
             (w.slab_case(nx=10, ny=10, nz=3, h=0.25), {"precision": ep.EP_FP64_PLAIN}, None),
             (w.slab_case(nx=12, ny=8, nz=3, h=0.25), {}, "bido")]

    def make():
        js = []
        for case, kw, extra in specs:
            j = ep.job_from_case(ctx, case, **kw)
            if extra == "bido":
                j.enable_bidomain(0.62 / 1.4, 0.24 / 1.4)
            js.append(j)
        return js
    alone = make()
    for j in alone:
        j.step(150)
    batch = make()
    ep.step(batch, 150)
    for a, b in zip(alone, batch):
        assert a.step_index == b.step_index == 150
        assert np.array_equal(a.V, b.V)
        assert np.array_equal(a.activation_times(), b.activation_times())
        for k in range(1, 19):
            assert np.array_equal(a.read(k), b.read(k))
    assert np.array_equal(alone[-1].ve, batch[-1].ve)
    ctx.close()


PLAIN_SHAPES = (0, 1, 2, 3, 4, 5, 10, 11)


@pytest.mark.parametrize("three_models", [False, True])
def test_one_job_kernels_equal_the_batched_kernels(three_models):
    """The kernels of an FP32 group take the jobs' descriptors as a kernel
    parameter: a one-job instance (the descriptor at a fixed place, the step
    counter read once) and a 15-job instance (each tile's job found from the
    group's tile bounds). For every two-launch shape, a job stepped alone is
    bitwise the same job stepped in a batch with another (TP06-only cells,
    and TP06 / Courtemanche / Stewart regions with two stimuli, ragged
    tiles)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    case = _three_model_case() if three_models else w.slab_case(nx=13, ny=9, nz=3, h=0.25, stim_x=0.6)
    other = w.slab_case(nx=7, ny=5, nz=3, h=0.5)
    ctx = ep.Context()
    for v in PLAIN_SHAPES:
        ep.set_cell_variant(ctx, ep.EP_FP32_MIXED, v)
        alone = ep.job_from_case(ctx, case)
        alone.step(250)
        a = ep.job_from_case(ctx, case)
        b = ep.job_from_case(ctx, other)
        ep.step([a, b], 250)
        for x, y in zip(_state(alone), _state(a)):
            assert np.array_equal(x, y, equal_nan=True), v
        assert np.isfinite(_state(alone)[-1]).any()
        for j in (alone, a, b):
            j.destroy()
    ctx.close()


def test_launch_groups_equal_alone():
    """A batch is stepped in launch groups: FP32 forward-Euler jobs at most 15
    to a group (descriptors as a kernel parameter), the other FP32 jobs (AB2
    here) in one group with the job table in global memory, the FP64 jobs in
    another. Twenty jobs of different sizes -- 17 forward Euler (groups of 15
    and 2), one AB2, two FP64 -- each end bitwise where they end stepped
    alone, with captured-graph replay and direct launches."""
    import torch
    assert torch.cuda.is_available()
    from paper_2112_12854_b300 import ep
    ctx = ep.Context()
    specs = [(w.slab_case(nx=5 + k % 6, ny=4 + k % 3, nz=3, h=0.5, stim_x=0.6), {}) for k in range(17)]
    specs.append((w.slab_case(nx=8, ny=6, nz=3, h=0.5), {"integrator": 1}))
    specs += [(w.slab_case(nx=7 + k, ny=5, nz=3, h=0.5), {"precision": ep.EP_FP64_PLAIN}) for k in range(2)]

    def make():
        return [ep.job_from_case(ctx, case, **kw) for case, kw in specs]
    alone = make()
    for j in alone:
        j.step(130)
    batch = make()
    ep.step(batch, 100)       # one captured graph of the whole batch
    ep.step(batch, 30)
    for a, b in zip(alone, batch):
        assert a.step_index == b.step_index == 130
        assert np.array_equal(a.V, b.V)
        assert np.array_equal(a.activation_times(), b.activation_times(), equal_nan=True)
        for k in range(1, 19):
            assert np.array_equal(a.read(k), b.read(k))
    assert sum(np.isfinite(a.activation_times()).any() for a in alone) >= 17
    ctx.close()
