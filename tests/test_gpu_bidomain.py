"""Parity of the CUDA bidomain path (Eq. 1, Eqs. 5-6: cell update with the
intracellular flux of V + v_e, then the elliptic equation for v_e by
restarted GMRES in one cooperative launch) with the FP64 oracle, through the
C ABI; plus the exact parallel-tensor reduction on the GPU, batching and
state I/O."""
import numpy as np
import pytest

import workloads as w
from gpu_common import act_error, tolerances

pytestmark = pytest.mark.gpu

# Table 2 (mS/mm) over chi C_m = 1.4 uF/mm^3: intracellular and extracellular
DIL, DIT = 0.17 / 1.4, 0.019 / 1.4
DEL, DET = 0.62 / 1.4, 0.24 / 1.4
TOL_VE = {"mixed": 0.1, "plain": 1e-6}


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


def _slab(cubes=(12, 8, 3), h=0.25, D=(DIL, DIT), models=(0,), fibre_rot=True):
    xyz, tets = w.kuhn_box(*cubes, h)
    n = tets.shape[0]
    c = w.tet_centroids(xyz, tets)
    fib = w.fibres_transmural(c[:, 2], 0.0, cubes[2] * h) if fibre_rot else w.fibres_uniform(n)
    ps = (np.arange(n) * len(models) // n).astype(np.uint8)
    sets = [w.ParamSet(model=m, D_l=D[0], D_t=D[1]) for m in models]
    return w.TissueCase("slab", xyz, tets, fib, ps, ((c[:, 0] < 0.6) & (c[:, 1] < 0.6)).astype(np.uint8),
                        sets, [w.Stimulus(-80.0, 0.0, 1.0)], 0.02, 0, -20.0)


@pytest.mark.parametrize("pname,reorth", [("mixed", 0), ("plain", 0), ("mixed", 1)])
def test_bidomain_parity(ctx, pname, reorth):
    """Mixed TP06 / Courtemanche / Stewart slab with rotating fibres and
    unequal anisotropy ratios; V, v_e and activation times against the
    oracle at three output times (1728 cells: several tiles, ragged tail),
    with Gram-Schmidt once (default) and twice."""
    import oracle
    from paper_2112_12854_b300 import ep
    prec = _prec(pname)
    tv, ta = tolerances(prec)
    case = _slab(models=(0, 1, 2))
    o = oracle.Sim(case)
    o.set_bidomain(DEL, DET, tol=1e-11)
    j = ep.job_from_case(ctx, case, precision=prec)
    j.enable_bidomain(DEL, DET, reorth=reorth)
    assert np.abs(j.ve - o.ve).max() <= TOL_VE[pname]
    done = 0
    for n in (100, 250, 500):
        o.run(n - done)
        j.step(n - done)
        done = n
        dv = np.abs(j.V - o.V).max()
        de = np.abs(j.ve - o.ve).max()
        print(pname, n, "max|dV|", dv, "max|dve|", de, j.bidomain_stats())
        assert dv <= tv and de <= TOL_VE[pname]
    assert np.isfinite(o.activation_times()).sum() > 100
    assert act_error(j.activation_times(), o.activation_times()) <= ta
    st = j.bidomain_stats()
    assert not st["failed"] and st["solves"] == 501
    j.destroy()


@pytest.mark.parametrize("pname", ["mixed", "plain"])
def test_bidomain_long_run_and_restart_of_the_initial_guess(ctx, pname):
    """The GPU solve starts from 2 v_e^n - v_e^{n-1} (the oracle from v_e^n).
    While the front moves, the extrapolated start needs fewer Arnoldi steps
    than the first solve after v_e is written from the host, which starts
    from v_e^n; over 2500 steps (50 ms: the front crosses the slab and the
    plateau begins) no solve fails and V and v_e stay within tolerance of
    the oracle."""
    import oracle
    from paper_2112_12854_b300 import ep
    prec = _prec(pname)
    tv, _ = tolerances(prec)
    case = _slab()
    o = oracle.Sim(case)
    o.set_bidomain(DEL, DET, tol=1e-11)
    j = ep.job_from_case(ctx, case, precision=prec)
    j.enable_bidomain(DEL, DET)
    j.step(60)
    t0 = j.bidomain_stats()["total_iters"]
    j.step(20)
    extrap = (j.bidomain_stats()["total_iters"] - t0) / 20
    j.ve = j.ve                                  # host write: the next solve starts from v_e^n
    j.step(1)
    first = j.bidomain_stats()["last_iters"]
    print(pname, "Arnoldi steps: extrapolated start", extrap, "first solve after a write", first)
    assert extrap < first
    done = 81
    o.run(done)
    for n in (500, 1500, 2500):
        o.run(n - done)
        j.step(n - done)
        done = n
        st = j.bidomain_stats()
        dv, de = np.abs(j.V - o.V).max(), np.abs(j.ve - o.ve).max()
        print(pname, n, "max|dV|", dv, "max|dve|", de, "mean Arnoldi steps", st["total_iters"] / st["solves"])
        assert not st["failed"] and np.isfinite(j.V).all() and np.isfinite(j.ve).all()
        assert dv <= tv and de <= TOL_VE[pname]
    j.destroy()


def test_parallel_tensors_reduce_to_monodomain_on_gpu(ctx):
    """M_e = lambda M_i: the GPU bidomain run equals the GPU monodomain run
    with M = lambda M_i / (1 + lambda) (FP64 plain, solver tolerance)."""
    from paper_2112_12854_b300 import ep
    lam = 2.0
    bi = ep.job_from_case(ctx, _slab(D=(DIL, DIT)), precision=ep.EP_FP64_PLAIN)
    bi.enable_bidomain(lam * DIL, lam * DIT, tol=1e-12)
    mo = ep.job_from_case(ctx, _slab(D=(lam / (1 + lam) * DIL, lam / (1 + lam) * DIT)), precision=ep.EP_FP64_PLAIN)
    for _ in range(3):
        bi.step(100)
        mo.step(100)
        assert np.abs(bi.V - mo.V).max() < 1e-7
        g = bi.ve + bi.V / (1 + lam)
        assert np.abs(g - g.mean()).max() < 1e-7
    bi.destroy()
    mo.destroy()


def test_bidomain_batched_bitwise_and_ve_io(ctx):
    """A bidomain job stepped in a batch with monodomain jobs gives the
    results it gives alone; v_e written back restores the run."""
    from paper_2112_12854_b300 import ep
    case = _slab(cubes=(10, 6, 2))

    def make():
        j = ep.job_from_case(ctx, case)
        j.enable_bidomain(DEL, DET)
        return j
    alone = make()
    alone.step(150)
    a1 = make()
    other = ep.job_from_case(ctx, w.slab_case(nx=7, ny=5, nz=2))
    ep.step([other, a1], 150)
    assert np.array_equal(a1.V, alone.V) and np.array_equal(a1.ve, alone.ve)
    # checkpoint / restore: state and v_e of `alone` copied into a fresh job
    nvar = len(ep.model_varnames(ep.EP_TP06))
    snap = [alone.read(v) for v in range(nvar)]
    ve = alone.ve
    b = make()
    for v in range(nvar):
        b.write(v, snap[v])
    b.ve = ve
    b.step_index = alone.step_index
    alone.step(50)
    b.step(50)
    assert np.abs(b.V - alone.V).max() < 1e-4
    for j in (alone, a1, b, other):
        j.destroy()


def test_barrier_wait_gives_up_and_other_jobs_are_unaffected(ctx):
    """The solve kernel's grid-barrier waits are bounded. With the bound set
    to 1 ns on a multi-block solve, a block that has to wait at all gives up:
    it raises the solve's error flag, every block leaves at its next barrier
    (the launch completes: the stream synchronises), and ep_bidomain_stats
    reports EP_ETIMEOUT. A second bidomain job stepped in the same batch is
    bitwise equal to the same job stepped alone, and once the first job's
    v_e is restored (which clears the record) and the default bound is back,
    its solves run normally again. No GPU fault is involved: the kernel
    returns an error status that the host reads."""
    from paper_2112_12854_b300 import ep
    case = _slab(cubes=(40, 30, 6))                      # 43200 cells: tens of blocks per solve
    bad = ep.job_from_case(ctx, case)
    good = ep.job_from_case(ctx, case)
    alone = ep.job_from_case(ctx, case)
    bad.enable_bidomain(DEL, DET, barrier_limit_s=1e-9)
    good.enable_bidomain(DEL, DET)
    alone.enable_bidomain(DEL, DET)
    ep.step([bad, good], 20)
    alone.step(20)
    import torch
    torch.cuda.synchronize()                             # every block of every solve has returned
    with pytest.raises(ep.EPError) as e:
        bad.bidomain_stats()
    assert e.value.code == ep.EP_ETIMEOUT
    st = good.bidomain_stats()
    assert not st["timeout"] and not st["failed"] and st["solves"] == 21
    assert np.array_equal(good.V, alone.V)
    assert np.array_equal(good.ve, alone.ve)
    # recovery: default bound, state and v_e restored from the healthy job
    bad.enable_bidomain(DEL, DET)
    for v in range(19):
        bad.write(v, alone.read(v))
    bad.step_index = alone.step_index
    bad.ve = alone.ve
    assert not bad.bidomain_stats()["timeout"]
    ep.step([bad], 10)
    alone.step(10)
    assert not bad.bidomain_stats()["timeout"]
    assert np.abs(bad.V - alone.V).max() < 1e-3
    for j in (bad, good, alone):
        j.destroy()
