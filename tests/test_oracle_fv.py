"""Pins of the oracle's mesh geometry and finite-volume diffusion operator
(Sec. 3.2, Eqs. 7-8) against what the mathematics fixes.

None of these tests re-evaluates the oracle's formulas: each checks a property
the exact operator must have (an invariant, an exactness class, a closed form
derived by hand, a convergence limit)."""
import os

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _interior(xyz, centroids, margin):
    lo, hi = xyz.min(0), xyz.max(0)
    return np.all((centroids > lo + margin) & (centroids < hi - margin), axis=1)


def _tensor_field(orc, m, fibre, D_l, D_t):
    return np.tile(orc.conductivity(fibre, D_l, D_t).ravel(), (m.n_cells, 1))


def test_table1_cell_counts_match_kuhn_split():
    """Table 1's cell counts are the 6-tet split of the 20x7x3 mm box."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_cell_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for dx, cells in rows:
        dx = float(dx)
        n = [round(L / dx) for L in (20.0, 7.0, 3.0)]
        assert 6 * n[0] * n[1] * n[2] == int(cells)
    xyz, tets = w.kuhn_box(40, 14, 6, 0.5)
    assert tets.shape[0] == 20160


def test_face_counts_and_neighbours(orc):
    xyz, tets = w.kuhn_box(16, 16, 4, 0.5)
    m = orc.Mesh(xyz, tets)
    assert m.n_nodes == 1445 and m.n_cells == 6144
    # boundary: 2 triangles per boundary square
    assert m.n_boundary_faces == 2 * 2 * (16 * 16 + 16 * 4 + 16 * 4)
    c, vol, nb = m.cell_info()
    assert np.allclose(vol, 0.5 ** 3 / 6)
    # neighbour relation is symmetric
    for cell in range(0, m.n_cells, 97):
        for k in range(4):
            o = nb[cell, k]
            if o >= 0:
                assert cell in nb[o]


def test_rejects_degenerate_and_nonmanifold(orc):
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [2, 2, 0], [0, 0, 1]], float)
    with pytest.raises(ValueError):
        orc.Mesh(xyz, np.array([[0, 1, 2, 3]], np.int32))          # flat tet
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1]], float)
    tets = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], np.int32)  # face shared 3x
    with pytest.raises(ValueError):
        orc.Mesh(xyz, tets)


def test_conductivity_tensor_eigenstructure(orc):
    """Eqs. 2-3: D has eigenvalue D_l along the fibre and D_t across it."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        f = rng.standard_normal(3)
        f /= np.linalg.norm(f)
        D = orc.conductivity(f, 0.154, 0.0385)
        assert np.allclose(D, D.T, atol=1e-15)
        assert np.allclose(D @ f, 0.154 * f, atol=1e-14)
        ev = np.sort(np.linalg.eigvalsh(D))
        assert np.allclose(ev, [0.0385, 0.0385, 0.154], atol=1e-14)


def test_conservation_and_row_sums(orc):
    """Each interior face flux leaves one cell and enters the other, so
    sum_c V_c (dV/dt)_c = 0 for any field; a constant field has no flux."""
    xyz, tets = w.kuhn_box(6, 5, 4, 0.5)
    m = orc.Mesh(xyz, tets)
    c, vol, _ = m.cell_info()
    rng = np.random.default_rng(0)
    fib = rng.standard_normal((m.n_cells, 3))
    D = m.tensors(fib, 0.154, 0.0385)
    for _ in range(3):
        v = rng.standard_normal(m.n_cells)
        out = m.diffusion(D, v)
        assert abs(np.sum(out * vol)) < 1e-13 * np.sum(np.abs(out * vol))
    assert np.abs(m.diffusion(D, np.full(m.n_cells, -85.0))).max() < 1e-12


def test_linear_patch_exact(orc):
    """The Kuhn mesh is centrally symmetric about every vertex, so for a linear
    field every interior stage is exact: node values, face values, Gauss-Green
    gradient (= a), interpolated face gradient, zero correction (Eq. 8), and a
    constant tensor gives zero divergence. A wrong sign of e, a wrong normal
    orientation or a wrong gradient weight breaks this."""
    xyz, tets = w.kuhn_box(8, 8, 8, 0.5)
    m = orc.Mesh(xyz, tets)
    c, vol, nb = m.cell_info()
    a = np.array([0.3, -0.7, 1.1])
    v = c @ a
    lo, hi = xyz.min(0), xyz.max(0)
    bnode = np.any((xyz < lo + 1e-9) | (xyz > hi - 1e-9), axis=1)
    touches = bnode[tets].any(1)
    nb2 = np.where(nb < 0, np.arange(m.n_cells)[:, None], nb)
    ring = touches | touches[nb2].any(1)
    vn = m.node_values(v)
    assert np.abs(vn[~bnode] - xyz[~bnode] @ a).max() < 1e-12
    g = m.cell_gradients(vn)
    assert np.abs(g[~touches] - a).max() < 1e-12
    D = _tensor_field(orc, m, [0.6, 0.8, 0.0], 0.154, 0.0385)
    out = m.diffusion(D, v)
    assert (~ring).sum() > 500
    assert np.abs(out[~ring]).max() < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_isotropic_quadratic_exact_per_cell(orc, axis):
    """With D = I, the discrete operator of x_k^2/2 is exactly 1 in every
    interior cell of the Kuhn mesh."""
    xyz, tets = w.kuhn_box(8, 8, 8, 0.5)
    m = orc.Mesh(xyz, tets)
    c, vol, _ = m.cell_info()
    D = np.tile(np.eye(3).ravel(), (m.n_cells, 1))
    out = m.diffusion(D, 0.5 * c[:, axis] ** 2)
    inner = _interior(xyz, c, 1.2)
    assert inner.sum() > 200
    assert np.abs(out[inner] - 1.0).max() < 1e-10


def test_anisotropic_quadratic_weak_consistency(orc):
    """For any quadratic q and constant tensor D, the interior volume average
    of the discrete operator equals div(D grad q) = sum_ij D_ij d_ij q, for
    random fibre directions (pins Eqs. 2-3 and the face tensor)."""
    xyz, tets = w.kuhn_box(10, 10, 10, 0.5)
    m = orc.Mesh(xyz, tets)
    c, vol, _ = m.cell_info()
    inner = _interior(xyz, c, 1.2)
    rng = np.random.default_rng(1)
    for _ in range(3):
        f = rng.standard_normal(3)
        f /= np.linalg.norm(f)
        Dm = orc.conductivity(f, 0.154, 0.0385)
        D = np.tile(Dm.ravel(), (m.n_cells, 1))
        for i, j in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
            q = c[:, i] * c[:, j] * (0.5 if i == j else 1.0)
            exact = Dm[i, j] * (1.0 if i == j else 2.0)
            out = m.diffusion(D, q)
            mean = np.sum((out * vol)[inner]) / np.sum(vol[inner])
            assert abs(mean - exact) < 1e-9


def test_two_tet_bipyramid_closed_form(orc):
    """Two tets sharing a face in z=0 (centroid at the origin), apexes at
    (0,0,+a) and (0,0,-a). By hand: shared nodes get (v1+v2)/2, apexes v1 and
    v2; both Gauss-Green gradients are (v1-v2)/(2a) z; alpha = 1/2, d = a/2,
    e = z, so Eq. 8 gives grad v_f = 2 (v1-v2)/a z and the outputs are
    -/+ 6 D_zz (v1 - v2) / a^2 (independent of the other tensor entries)."""
    a = 0.7
    P = np.array([[1.0, 0.2, 0.0], [-0.4, 0.9, 0.0], [-0.6, -1.1, 0.0]])
    xyz = np.vstack([P, [[0, 0, a], [0, 0, -a]]])
    tets = np.array([[0, 1, 2, 3], [0, 2, 1, 4]], np.int32)
    m = orc.Mesh(xyz, tets)
    Dm = np.array([[0.3, 0.05, 0.02], [0.05, 0.2, -0.04], [0.02, -0.04, 0.11]])
    D = np.tile(Dm.ravel(), (2, 1))
    v1, v2 = -80.0, 12.5
    out = m.diffusion(D, np.array([v1, v2]))
    ref = 6.0 * Dm[2, 2] * (v1 - v2) / a ** 2
    assert np.allclose(out, [-ref, ref], rtol=1e-12)
    vn = m.node_values(np.array([v1, v2]))
    assert np.allclose(vn, [(v1 + v2) / 2] * 3 + [v1, v2], rtol=1e-13)


def test_single_tet_has_no_flux(orc):
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    m = orc.Mesh(xyz, np.array([[0, 1, 2, 3]], np.int32))
    assert m.diffusion(np.eye(3).ravel()[None], np.array([3.0]))[0] == 0.0


def test_twopoint_part_symmetric(orc):
    """The two-point part of the flux, volume-weighted, is a symmetric matrix;
    the full wide-stencil operator is not in general (its asymmetry is
    reported, not asserted)."""
    xyz, tets = w.kuhn_box(3, 2, 2, 0.5)
    m = orc.Mesh(xyz, tets)
    c, vol, _ = m.cell_info()
    rng = np.random.default_rng(5)
    D = m.tensors(rng.standard_normal((m.n_cells, 3)), 0.154, 0.0385)
    n = m.n_cells
    L2 = np.stack([m.diffusion(D, np.eye(n)[k], twopoint=True) for k in range(n)], axis=1)
    A = vol[:, None] * L2
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    L = np.stack([m.diffusion(D, np.eye(n)[k]) for k in range(n)], axis=1)
    Af = vol[:, None] * L
    asym = np.linalg.norm(Af - Af.T) / np.linalg.norm(Af)
    assert 0.0 <= asym < 1.0


def _rayleigh(orc, n, fibre):
    h = 0.5 / n
    nx, ny, nz = 8 * n, 2 * n, 2 * n
    xyz, tets = w.kuhn_box(nx, ny, nz, h)
    m = orc.Mesh(xyz, tets)
    c, vol, _ = m.cell_info()
    k = np.pi / (nx * h)
    D = _tensor_field(orc, m, fibre, 0.154, 0.0385)
    v = np.cos(k * c[:, 0])
    out = m.diffusion(D, v)
    return -np.sum(out * v * vol) / np.sum(v * v * vol), k


@pytest.mark.parametrize("theta", [0.0, 0.5, np.pi / 2])
def test_cosine_mode_decay_rate_converges(orc, theta):
    """cos(pi x / L) satisfies the zero-flux condition; its decay rate under
    the discrete operator (Rayleigh quotient) converges to
    (D_l cos^2 th + D_t sin^2 th) k^2 under refinement."""
    fib = [np.cos(theta), np.sin(theta), 0.0]
    errs = []
    for n in (1, 2, 4):
        lam, k = _rayleigh(orc, n, fib)
        exact = (0.154 * np.cos(theta) ** 2 + 0.0385 * np.sin(theta) ** 2) * k * k
        errs.append(abs(lam / exact - 1.0))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.04
