"""Pins of the oracle's bidomain step (Eq. 1, Eqs. 5-6): the extracellular
potential from the elliptic equation by restarted GMRES.

- With parallel tensors, M_e = lambda M_i, the bidomain reduces exactly to
  the monodomain with M = lambda M_i / (1 + lambda) (Sec. 3.2, Eq. 6 to
  Eq. 7): the V trajectories agree to solver precision and
  v_e = -V / (1 + lambda) + const.
- The GMRES solution equals a dense least-squares solve of the assembled
  operators (numpy) on a tiny mesh, in the zero-mean gauge.
- A plane wave along the fibres sees the half harmonic mean of the
  longitudinal conductivities (the monodomain approximation of Sec. 1):
  its activation times match that monodomain run closely.
"""
import numpy as np

import workloads as w


def _case(cubes, h, D_l, D_t, stim_x=0.5, amp=-80.0, fibre=None):
    xyz, tets = w.kuhn_box(*cubes, h)
    n = tets.shape[0]
    c = w.tet_centroids(xyz, tets)
    return w.TissueCase("slab", xyz, tets, w.fibres_uniform(n) if fibre is None else fibre,
                        np.zeros(n, np.uint8), (c[:, 0] < stim_x).astype(np.uint8),
                        [w.ParamSet(model=0, D_l=D_l, D_t=D_t)], [w.Stimulus(amp, 0.0, 1.0)], 0.02, 0, -20.0)


def test_parallel_tensors_reduce_to_monodomain(orc):
    Dl, Dt, lam = 0.12, 0.03, 2.5
    bi = orc.Sim(_case((10, 6, 2), 0.25, Dl, Dt))
    bi.set_bidomain(lam * Dl, lam * Dt, tol=1e-11)
    mo = orc.Sim(_case((10, 6, 2), 0.25, lam / (1 + lam) * Dl, lam / (1 + lam) * Dt))
    for _ in range(3):
        bi.run(60)
        mo.run(60)
        assert np.abs(bi.V - mo.V).max() < 1e-7
        g = bi.ve + bi.V / (1 + lam)
        assert np.abs(g - g.mean()).max() < 1e-7
    assert np.isfinite(mo.activation_times()).any()       # a wave is moving
    st = bi.bidomain_stats()
    assert not st["failed"] and st["last_rel_res"] <= 1e-11


def test_gmres_matches_dense_solve(orc):
    """v_e from the oracle's GMRES against numpy's least-squares solution of
    the assembled L_ie x = -L_i V (operators assembled column by column from
    the diffusion operator, the sum of tensors D_i + D_e formed here)."""
    rng = np.random.default_rng(3)
    case = _case((3, 2, 2), 0.5, 0.1, 0.02)
    n = case.n_cells
    s = orc.Sim(case)
    V = rng.uniform(-85.0, 20.0, n)
    s.set(0, V)
    Del, Det = 0.3, 0.15
    s.set_bidomain(Del, Det, tol=1e-13)
    m = orc.Mesh(case.xyz, case.tets)
    Di = m.tensors(case.fibre, 0.1, 0.02)
    Die = Di + m.tensors(case.fibre, Del, Det)
    eye = np.eye(n)
    Ai = np.stack([m.diffusion(Di, eye[k]) for k in range(n)], axis=1)
    Aie = np.stack([m.diffusion(Die, eye[k]) for k in range(n)], axis=1)
    x, *_ = np.linalg.lstsq(Aie, -Ai @ V, rcond=None)
    _, vol, _ = m.cell_info()
    x -= np.dot(vol, x) / vol.sum()
    ve = s.ve
    assert abs(np.dot(vol, ve)) < 1e-10 * vol.sum()
    assert np.abs(ve - x).max() < 1e-8 * max(1.0, np.abs(x).max())
    # the residual of the elliptic equation, by the oracle's own operator
    r = s.bidomain_operator(ve) + m.diffusion(Di, V)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(Ai @ V)


def test_plane_wave_sees_harmonic_mean(orc):
    """Unequal anisotropy ratios (Table 2's intra/extracellular values): a
    plane wave along the fibres propagates as the monodomain with the
    longitudinal half harmonic mean of the two conductivities."""
    Dil, Dit = 0.17 / 1.4, 0.019 / 1.4
    Del, Det = 0.62 / 1.4, 0.24 / 1.4
    hl, ht = Dil * Del / (Dil + Del), Dit * Det / (Dit + Det)
    cubes = (24, 2, 2)
    bi = orc.Sim(_case(cubes, 0.25, Dil, Dit))
    bi.set_bidomain(Del, Det, tol=1e-9)
    mo = orc.Sim(_case(cubes, 0.25, hl, ht))
    bi.run(600)
    mo.run(600)
    xyz, tets = w.kuhn_box(*cubes, 0.25)
    cx = w.tet_centroids(xyz, tets)[:, 0]
    far = cx > 5.0
    ta, tm = bi.activation_times()[far], mo.activation_times()[far]
    assert np.isfinite(tm).all() and np.isfinite(ta).all()
    assert np.abs(ta - tm).max() <= 0.01 * tm.max()
