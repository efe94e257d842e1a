"""Dense brute-force check of the oracle's diffusion operator on meshes of a
few tetrahedra (Sec. 3.2, Eqs. 7-8): the operator's matrix, obtained by
applying the oracle to every unit vector, against a second evaluation
written here in numpy straight from the geometric definitions, as dense
stage matrices (node averaging, Gauss-Green gradient, face gradient with
the Eq. 8 correction, face flux).

The meshes are the Kuhn split of one cube (6 tetrahedra, every node on the
boundary, interior faces only between tetrahedra of the cube) and of two
cubes side by side (12 tetrahedra: interior faces inside each cube and
across their shared square), with jittered nodes so that no weight is
symmetric (alpha != 1/2, unequal inverse distances) and a different
anisotropic tensor in every cell. Boundary faces carry no flux."""
import numpy as np
import pytest

import workloads as w


def _tet_geometry(xyz, tets):
    X = xyz[tets]                                            # (N, 4, 3)
    xc = X.mean(axis=1)
    vol = np.abs(np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6
    return X, xc, vol


def dense_operator(xyz, tets, Dc):
    """Matrix L (N x N) with (L v)_c = (1/V_c) sum_f A_f (D_f grad v_f) . n_f."""
    N, Nn = tets.shape[0], xyz.shape[0]
    X, xc, vol = _tet_geometry(xyz, tets)
    # S1: inverse-distance node averages, vn = P v
    Wt = np.zeros((Nn, N))
    for c in range(N):
        for k in tets[c]:
            Wt[k, c] = 1.0 / np.linalg.norm(xyz[k] - xc[c])
    P = Wt / Wt.sum(axis=1, keepdims=True)
    # faces: the face opposite local vertex i, with its outward area vector
    faces = {}
    G = np.zeros((N, 3, Nn))                                 # grad_c = G[c] @ vn  (S2, Gauss-Green)
    outward = {}
    for c in range(N):
        for i in range(4):
            f = [int(tets[c, j]) for j in range(4) if j != i]
            a = 0.5 * np.cross(xyz[f[1]] - xyz[f[0]], xyz[f[2]] - xyz[f[0]])
            if np.dot(a, xyz[f].mean(axis=0) - xc[c]) < 0:
                a = -a
            outward[(c, i)] = a
            for k in f:                                      # v_f = mean of the face's three node values
                G[c, :, k] += a / (3.0 * vol[c])
            faces.setdefault(tuple(sorted(f)), []).append((c, i))
    Gv = np.einsum("cdk,kn->cdn", G, P)                      # grad_c = Gv[c] @ v
    L = np.zeros((N, N))
    for key, sides in faces.items():
        if len(sides) == 1:
            continue                                         # boundary face: zero flux
        (c1, i1), (c2, _) = sides
        xf = xyz[list(key)].mean(axis=0)
        r1, r2 = np.linalg.norm(xc[c1] - xf), np.linalg.norm(xc[c2] - xf)
        a1, a2 = r2 / (r1 + r2), r1 / (r1 + r2)
        d = np.linalg.norm(xc[c1] - xc[c2])
        e = (xc[c1] - xc[c2]) / d
        gbar = a1 * Gv[c1] + a2 * Gv[c2]                     # (3, N): interpolated face gradient
        dvde = np.zeros(N)
        dvde[c1], dvde[c2] = 1.0 / d, -1.0 / d               # (v_c1 - v_c2) / d
        gf = gbar + np.outer(e, dvde - e @ gbar)             # Eq. 8: directional derivative along e replaced
        Df = a1 * Dc[c1] + a2 * Dc[c2]
        flux = (Df @ gf).T @ outward[(c1, i1)]               # out of c1, as a row over v
        L[c1] += flux / vol[c1]
        L[c2] -= flux / vol[c2]
    return L


def _case(nx, seed):
    xyz, tets = w.kuhn_box(nx, 1, 1, 0.5)
    rng = np.random.default_rng(seed)
    xyz = xyz + rng.uniform(-0.06, 0.06, xyz.shape)
    N = tets.shape[0]
    f = rng.standard_normal((N, 3))
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    Dl, Dt = rng.uniform(0.1, 0.2, N), rng.uniform(0.01, 0.05, N)
    Dc = np.stack([Dt[c] * np.eye(3) + (Dl[c] - Dt[c]) * np.outer(f[c], f[c]) for c in range(N)])
    return xyz, tets, Dc


@pytest.mark.parametrize("nx,seed", [(1, 11), (2, 12), (2, 13)])
def test_dense_operator_equals_geometric_evaluation(orc, nx, seed):
    xyz, tets, Dc = _case(nx, seed)
    N = tets.shape[0]
    assert N == 6 * nx
    m = orc.Mesh(xyz, tets)
    _, vol_o, nb = m.cell_info()
    _, _, vol = _tet_geometry(xyz, tets)
    assert np.allclose(vol_o, vol, rtol=1e-14)
    eye = np.eye(N)
    L_orc = np.stack([m.diffusion(Dc.reshape(N, 9), eye[k]) for k in range(N)], axis=1)
    L_ref = dense_operator(xyz, tets, Dc)
    scale = np.abs(L_ref).max()
    assert scale > 0
    assert np.abs(L_orc - L_ref).max() < 1e-12 * scale
    # every cell of the cube meets others (all entries of a row are used), and
    # the cells across the shared square of the two cubes are coupled
    assert np.all(np.count_nonzero(np.abs(L_ref) > 1e-12 * scale, axis=1) >= 3)
    if nx == 2:
        assert np.abs(L_ref[:6, 6:]).max() > 1e-6 * scale

