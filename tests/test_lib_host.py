"""Host-side checks of the CUDA library that need no GPU: the shared library
loads and exports the C ABI, and its planner's folded FP64 operator equals
the oracle's face-by-face evaluation of Eqs. 7-8 (an identity, not shared
code: the planner folds S1-S3 into per-cell coefficients independently)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as w
from paper_2112_12854_b300 import ep

HDR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ep.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ep_[a-z_0-9]+)\s*\(", src)) - {"ep_alloc_fn", "ep_free_fn"})


def test_library_exports_every_declared_symbol():
    L = ep.load()
    names = _declared()
    assert "ep_step" in names and "ep_mesh_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(ep.EXPORTS)


def test_model_variable_tables():
    assert len(ep.model_varnames(ep.EP_TP06)) == 19
    assert len(ep.model_varnames(ep.EP_CRN)) == 21
    assert len(ep.model_varnames(ep.EP_STEWART)) == 20
    import oracle
    for m in range(3):
        assert ep.model_varnames(m) == oracle.model_varnames(m)


def test_compensated_variables_are_the_slow_concentrations():
    """The variables an FP32 job keeps as compensated sums (and transfers in
    FP64 only) are exactly [Na]i, [K]i and the SR calcium of each model;
    everything else, V included, is stored in the compute type."""
    expect = {ep.EP_TP06: {"Na_i", "K_i", "Ca_SR"}, ep.EP_STEWART: {"Na_i", "K_i", "Ca_SR"},
              ep.EP_CRN: {"Na_i", "K_i", "Ca_up", "Ca_rel"}}
    L = ep.load()
    for m, names in expect.items():
        comp = ep.model_var_compensated(m)
        assert {n for n, c in zip(ep.model_varnames(m), comp) if c} == names
        assert not comp[0]
        assert L.ep_model_var_compensated(m, len(comp)) == -1 and L.ep_model_var_compensated(m, -1) == -1
    assert L.ep_model_var_compensated(3, 0) == -1


def _params(sets, dt=0.02):
    return ep.make_params(dt, sets, [])


def _apply(plan, V):
    n = V.size
    vn = np.add.reduceat(plan["nw"] * V[plan["n2c"]], plan["n2c_ptr"][:-1]) if plan["n2c"].size else None
    # reduceat of empty rows returns the next value: guard rows with no cells
    empty = plan["n2c_ptr"][1:] == plan["n2c_ptr"][:-1]
    vn[empty] = 0.0
    tet, opp, nbr = plan["tet"].reshape(n, 4), plan["opp"].reshape(n, 4), plan["nbr"].reshape(n, 4)
    wa, wb, q = plan["wa"].reshape(n, 4), plan["wb"].reshape(n, 4), plan["q"].reshape(n, 4)
    out = (wa * vn[tet]).sum(1)
    out += np.where(opp >= 0, wb * vn[np.maximum(opp, 0)], 0.0).sum(1)
    out += np.where(nbr >= 0, q * (V[np.maximum(nbr, 0)] - V[:, None]), 0.0).sum(1)
    return out


def _compare(xyz, tets, fibre, sets, pset, seed=0):
    import oracle
    plan = ep.plan_inspect(xyz, tets, _params(sets), param_set=pset, fibre=fibre)
    order = plan["cell_order"]
    assert np.array_equal(np.sort(order), np.arange(tets.shape[0]))
    m = oracle.Mesh(xyz, tets)
    D = np.stack([oracle.conductivity(fibre[c], sets[pset[c]].D_l, sets[pset[c]].D_t).ravel()
                  for c in range(tets.shape[0])])
    rng = np.random.default_rng(seed)
    for _ in range(3):
        v = rng.uniform(-90, 40, tets.shape[0])
        ref = m.diffusion(D, v)
        got = np.empty_like(ref)
        got[order] = _apply(plan, v[order])
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() < 1e-11 * scale
    return plan


def test_folded_operator_equals_face_by_face_kuhn():
    xyz, tets = w.kuhn_box(6, 5, 3, 0.25)
    rng = np.random.default_rng(1)
    fib = rng.standard_normal((tets.shape[0], 3))
    sets = [w.ParamSet(D_l=0.154, D_t=0.0385), w.ParamSet(D_l=0.0953, D_t=0.0126)]
    pset = rng.integers(0, 2, tets.shape[0]).astype(np.uint8)
    _compare(xyz, tets, fib, sets, pset)


def test_folded_operator_equals_face_by_face_jittered_and_inverted():
    """A jittered (non-symmetric) mesh with randomly inverted tets and
    shuffled numbering exercises the alpha weights, the orientation fix and
    the renumbering."""
    xyz, tets = w.kuhn_box(5, 4, 4, 0.5)
    rng = np.random.default_rng(2)
    xyz = xyz + rng.uniform(-0.08, 0.08, xyz.shape)
    flip = rng.uniform(size=tets.shape[0]) < 0.5
    tets = tets.copy()
    tets[flip] = tets[flip][:, [0, 2, 1, 3]]
    perm = rng.permutation(tets.shape[0])
    tets = tets[perm]
    nperm = rng.permutation(xyz.shape[0])
    inv = np.argsort(nperm)
    xyz = xyz[nperm]
    tets = inv[tets].astype(np.int32)
    fib = rng.standard_normal((tets.shape[0], 3))
    _compare(xyz, tets, fib, [w.ParamSet()], np.zeros(tets.shape[0], np.uint8))


def test_rcm_reduces_bandwidth_and_groups_models():
    xyz, tets = w.kuhn_box(12, 6, 3, 0.5)
    rng = np.random.default_rng(3)
    perm = rng.permutation(tets.shape[0])
    tets = tets[perm]
    models = rng.integers(0, 3, tets.shape[0]).astype(np.uint8)
    plan = ep.plan_inspect(xyz, tets, _params([w.ParamSet()]), cell_model=models)
    order = plan["cell_order"]
    assert np.all(np.diff(models[order].astype(int)) >= 0)          # model-major
    plan1 = ep.plan_inspect(xyz, tets, _params([w.ParamSet()]))
    nbr = plan1["nbr"].reshape(-1, 4)
    c = np.repeat(np.arange(nbr.shape[0]), 4)
    bw_rcm = np.abs(nbr.ravel() - c)[nbr.ravel() >= 0].max()
    import oracle
    _, _, nb0 = oracle.Mesh(xyz, tets).cell_info()
    bw0 = np.abs(nb0.ravel() - np.repeat(np.arange(nb0.shape[0]), 4))[nb0.ravel() >= 0].max()
    assert bw_rcm < bw0 / 4


def test_gershgorin_bounds_spectrum():
    xyz, tets = w.kuhn_box(4, 3, 3, 0.25)
    plan = ep.plan_inspect(xyz, tets, _params([w.ParamSet()]), fibre=w.fibres_uniform(tets.shape[0]))
    n = tets.shape[0]
    L = np.stack([_apply(plan, np.eye(n)[k]) for k in range(n)], axis=1)
    rho = np.abs(np.linalg.eigvals(L)).max()
    assert rho <= plan["rho_bound"] * (1 + 1e-12)
    assert plan["rho_bound"] < 2.0 * rho


@pytest.mark.parametrize("case", ["degenerate", "range", "nonmanifold"])
def test_planner_rejects_bad_meshes(case):
    if case == "degenerate":
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float)
        tets = np.array([[0, 1, 2, 3]])
    elif case == "range":
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
        tets = np.array([[0, 1, 2, 7]])
    else:
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1]], float)
        tets = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]])
    with pytest.raises(ep.EPError) as e:
        ep.plan_inspect(xyz, tets, _params([w.ParamSet()]))
    assert e.value.code == ep.EP_EMESH


@pytest.mark.parametrize("n_cells,n_nodes", [(0, 4), (1 << 31, 4), (1, 1 << 31)])
def test_planner_rejects_empty_and_oversized_meshes(n_cells, n_nodes):
    """Cell and node indices are 32-bit on the device: an empty mesh and one
    with 2^31 cells or nodes are refused with EP_EINVAL before any array is
    read or allocated (the descriptor's arrays here are far too short)."""
    xyz = np.zeros((4, 3))
    tet = np.zeros((1, 4), np.int32)
    d = ep.MeshDesc()
    d.n_nodes, d.xyz, d.n_cells, d.tet = n_nodes, xyz.ctypes.data, n_cells, tet.ctypes.data
    d.n_tris, d.tri = 0, None
    for name in ("cell_model", "param_set", "stim_mask", "fibre"):
        setattr(d, name, None)
    prm = _params([w.ParamSet()])
    out = ctypes.c_void_p()
    L = ep.load()
    rc = L.ep_plan_create(ctypes.byref(d), ctypes.byref(prm), ctypes.byref(out))
    assert rc == ep.EP_EINVAL and not out.value
    msg = L.ep_last_error(None).decode()
    assert ("empty" in msg) if n_cells == 0 else ("2^31" in msg)


def test_planner_rejects_missing_param_set():
    xyz, tets = w.kuhn_box(2, 2, 2, 0.5)
    with pytest.raises(ep.EPError) as e:
        ep.plan_inspect(xyz, tets, _params([w.ParamSet()]), param_set=np.full(tets.shape[0], 3, np.uint8))
    assert e.value.code == ep.EP_EINVAL


def test_library_has_no_unresolved_internal_symbols():
    import subprocess
    out = subprocess.run(["nm", "-D", "--undefined-only", ep.LIB_PATH], capture_output=True, text=True).stdout
    bad = [l for l in out.splitlines() if "_ZN2ep" in l]
    assert not bad, bad


def test_ab2_halves_the_explicit_stability_bound():
    """AB2's stability interval on the negative real axis is [-1, 0], half
    forward Euler's [-2, 0]: a dt that forward Euler accepts on this mesh is
    rejected for AB2 (EP_EUNSTABLE) until it is halved (host-only planner)."""
    xyz, tets = w.kuhn_box(12, 8, 3, 0.25)
    n = tets.shape[0]
    for dt, integ, ok in ((0.02, 0, True), (0.02, 1, False), (0.01, 1, True)):
        case = w.TissueCase("slab", xyz, tets, w.fibres_uniform(n), np.zeros(n, np.uint8), np.zeros(n, np.uint8),
                            [w.ParamSet()], [], dt, 0, -20.0)
        if ok:
            ep.plan_from_case(case, integrator=integ).destroy()
        else:
            with pytest.raises(ep.EPError) as e:
                ep.plan_from_case(case, integrator=integ)
            assert e.value.code == ep.EP_EUNSTABLE


def test_folded_operator_on_shell_triangles_equals_oracle():
    """A job with tets and a curved, jittered Purkinje shell: the planner's
    folded operator on the triangles equals the oracle's edge-by-edge shell
    operator (fv2d), and on the tets the face-by-face one; the two media
    share no face."""
    import oracle
    xyz_t, tets = w.kuhn_box(4, 3, 2, 0.5)
    xyz_s, tris = w.tri_cylinder(12, 6, 4.0, 3.0)
    rng = np.random.default_rng(4)
    xyz_s = xyz_s + rng.uniform(-0.05, 0.05, xyz_s.shape)
    xyz = np.concatenate([xyz_t, xyz_s + [0.0, 0.0, 5.0]])
    tris = (tris + len(xyz_t)).astype(np.int32)
    nt, ns = len(tets), len(tris)
    fib = rng.standard_normal((nt + ns, 3))
    sets = [w.ParamSet(D_l=0.154, D_t=0.0385), w.ParamSet(D_l=2.82, D_t=1.3)]
    pset = np.concatenate([np.zeros(nt, np.uint8), np.ones(ns, np.uint8)])
    plan = ep.plan_inspect(xyz, tets, _params(sets), param_set=pset, fibre=fib, tris=tris)
    order = plan["cell_order"]
    assert np.array_equal(np.sort(order), np.arange(nt + ns))
    m, sh = oracle.Mesh(xyz_t, tets), oracle.Shell(xyz, tris)
    D = np.stack([oracle.conductivity(fib[c], sets[pset[c]].D_l, sets[pset[c]].D_t).ravel() for c in range(nt + ns)])
    for _ in range(3):
        v = rng.uniform(-90, 40, nt + ns)
        ref = np.concatenate([m.diffusion(D[:nt], v[:nt]), sh.diffusion(D[nt:], v[nt:])])
        got = np.empty_like(ref)
        got[order] = _apply(plan, v[order])
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    # no folded coefficient links a triangle to a tet
    nbr = plan["nbr"].reshape(-1, 4)
    is_tri = np.isin(order, np.arange(nt, nt + ns))
    for c in range(nt + ns):
        for k in range(4):
            if nbr[c, k] >= 0:
                assert is_tri[nbr[c, k]] == is_tri[c]


def _coned_sphere(levels):
    """Tets coning every triangle of a subdivided octahedron to the centre:
    one node shared by every cell (its node -> cell entries span the whole
    numbering), neighbours only across the cone sides."""
    v = [np.array(p, float) for p in ([1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1])]
    tris = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4), (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    for _ in range(levels):
        mid, new = {}, []

        def m(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                mid[k] = len(v) - 1
            return mid[k]
        for a, b, c in tris:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = new
    xyz = np.vstack(v + [np.zeros(3)]) * 5.0
    tets = np.array([(a, b, c, len(v)) for a, b, c in tris], np.int32)
    return xyz, tets


def test_index_width_chosen_by_the_numbering():
    """By default 16-bit cell gathers and a 32-bit node -> cell table; with
    index_width 16 both 16-bit where every offset fits (a slab); on a
    150 x 150 x 30-cube wedge (4.05M cells, RCM neighbour bandwidth about
    12.5k cells) 16-bit cell gathers but 32-bit node -> cell entries (the
    cells around one node span about six RCM levels, 75k cells); 32-bit
    everywhere where a node is shared by 131072 cells (its cells span the
    whole numbering, and so do the nodes of a run of cells next to it); and
    32-bit on request."""
    params = ep.make_params(0.01, [w.ParamSet()])
    case = w.slab_case(nx=20, ny=10, nz=4, h=0.5)
    p = ep.Plan(case.xyz, case.tets, params)
    assert (p.index_width, p.node_index_width) == (16, 32)          # the default: 16-bit cell gathers
    p = ep.Plan(case.xyz, case.tets, params, index_width=16)
    assert (p.index_width, p.node_index_width) == (16, 16)
    p = ep.Plan(case.xyz, case.tets, params, index_width=32)
    assert (p.index_width, p.node_index_width) == (32, 32)
    xyz, tets = _coned_sphere(7)            # (no parameters: only the mesh is planned)
    assert tets.shape[0] == 131072
    p = ep.Plan(xyz, tets, index_width=16)
    assert (p.index_width, p.node_index_width) == (32, 32)
    wedge = w.wedge_case(nx=150, ny=150, nz=30, h=0.25)
    p = ep.Plan(wedge.xyz, wedge.tets, index_width=16)
    assert (p.index_width, p.node_index_width) == (16, 32)
    p = ep.Plan(*_coned_sphere(5), index_width=16)
    assert (p.index_width, p.node_index_width) == (16, 16)
    with pytest.raises(ep.EPError) as e:
        ep.Plan(case.xyz, case.tets, params, index_width=8)
    assert e.value.code == ep.EP_EINVAL
