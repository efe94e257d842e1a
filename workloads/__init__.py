"""Seeded synthetic inputs shaped like the paper's workloads.

This module produces *inputs only*: node coordinates, tetrahedra, fibre
directions, per-cell parameter-set labels, stimulus-region masks and job mixes.
It holds none of the method's arithmetic (no geometry coefficients, no
diffusion operator, no cell model), so it can feed both the FP64 oracle and the
CUDA path without coupling them.

Mesh family: the paper's convergence benchmark is a Cartesian box split into
tetrahedra (Sec. 4, the 20x7x3 mm slab at 0.5/0.2/0.1 mm whose cell counts in
Table 1 equal 6 tets per cube). Each cube is split into the 6 tetrahedra of the
Kuhn (Freudenthal) triangulation: one tet per permutation of the axes, walking
from the cube's low corner to its high corner. All cubes use the same split, so
the mesh is conforming.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field, replace

import numpy as np

MASTER_SEED = 2112_12854

# Parameter-set labels used by the generators (the library and the oracle take
# the per-set parameters as explicit inputs; these are only conventional ids).
PS_EPI, PS_MID, PS_ENDO, PS_ISCHEMIC = 0, 1, 2, 3

_KUHN_PERMS = list(itertools.permutations(range(3)))


def kuhn_box(nx: int, ny: int, nz: int, h: float,
             origin=(0.0, 0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """Kuhn 6-tet split of an nx x ny x nz block of cubes of side h (mm).

    Returns (xyz [n_nodes,3] float64, tets [6*nx*ny*nz,4] int32). Nodes are
    numbered x-fastest; cells are cube-major (x-fastest cubes), 6 tets per cube
    in permutation order. Every tet is positively oriented.
    """
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1),
                             np.arange(nz + 1), indexing="ij")
    xyz = np.stack([ii.ravel(order="F"), jj.ravel(order="F"),
                    kk.ravel(order="F")], axis=1).astype(np.float64) * h
    xyz += np.asarray(origin, dtype=np.float64)

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    ci, cj, ck = (a.ravel(order="F") for a in (ci, cj, ck))
    n_cubes = ci.size
    tets = np.empty((n_cubes, 6, 4), dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        pos = [ci.copy(), cj.copy(), ck.copy()]
        verts = [nid(*pos)]
        for ax in perm:
            pos[ax] = pos[ax] + 1
            verts.append(nid(*pos))
        # odd permutations give negatively oriented tets: swap two vertices
        parity = sum(1 for a in range(3) for b in range(a + 1, 3)
                     if perm[a] > perm[b]) % 2
        if parity:
            verts[2], verts[3] = verts[3], verts[2]
        tets[:, t, :] = np.stack(verts, axis=1)
    return xyz, tets.reshape(-1, 4).astype(np.int32)


def tri_box(nx: int, ny: int, h: float, origin=(0.0, 0.0, 0.0)):
    """Flat rectangle of nx x ny squares of side h in the z = origin[2] plane,
    each split into two triangles along the same diagonal (the 2D Kuhn
    split: every interior node has six triangles, centrally symmetric).
    Returns (xyz [n_nodes, 3], tris [2 nx ny, 3] int32)."""
    ox, oy, oz = origin
    gx, gy = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    xyz = np.stack([ox + h * gx.ravel(), oy + h * gy.ravel(), np.full(gx.size, oz)], axis=1).astype(np.float64)
    nid = lambda i, j: i * (ny + 1) + j
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    i, j = i.ravel(), j.ravel()
    a, b, c, d = nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)
    tris = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]).astype(np.int32)
    return xyz, tris


def tri_cylinder(n_theta: int, n_z: int, radius: float, height: float, arc: float = np.pi):
    """A curved shell: the part of a cylinder of the given radius spanning
    `arc` radians and `height` mm, split like tri_box."""
    xyz, tris = tri_box(n_theta, n_z, 1.0)
    th = xyz[:, 0] / n_theta * arc
    z = xyz[:, 1] / n_z * height
    return np.stack([radius * np.cos(th), radius * np.sin(th), z], axis=1), tris


def tri_centroids(xyz: np.ndarray, tris: np.ndarray) -> np.ndarray:
    return xyz[tris].mean(axis=1)


def tet_centroids(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Vertex mean of each tet; used only to select input regions."""
    return xyz[tets].mean(axis=1)


def fibres_uniform(n_cells: int, direction=(1.0, 0.0, 0.0)) -> np.ndarray:
    f = np.asarray(direction, dtype=np.float64)
    f = f / np.linalg.norm(f)
    return np.tile(f, (n_cells, 1))


def fibres_transmural(centroid_z: np.ndarray, z_endo: float, z_epi: float,
                      angle_endo_deg: float = -60.0,
                      angle_epi_deg: float = 60.0) -> np.ndarray:
    """Fibre angle rotating linearly with normalised depth d from the
    endocardium, alpha(d) = angle_endo + (angle_epi - angle_endo) d, fibres in
    the x-y plane: f = (cos alpha, sin alpha, 0)."""
    d = np.clip((centroid_z - z_endo) / (z_epi - z_endo), 0.0, 1.0)
    a = np.deg2rad(angle_endo_deg + (angle_epi_deg - angle_endo_deg) * d)
    return np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], axis=1)


@dataclass
class Stimulus:
    """A stimulus protocol (Eq. 4): amplitude in uA/uF (negative depolarises),
    onset, duration and period in ms (period 0 = a single pulse)."""
    amplitude: float
    t_on: float
    duration: float
    period: float = 0.0


@dataclass
class ParamSet:
    """Per-parameter-set inputs. model: 0 = TP06, 1 = Courtemanche,
    2 = Stewart. variant (TP06): 0 epi, 1 mid, 2 endo. D_l, D_t in mm^2/ms."""
    model: int = 0
    variant: int = 0
    D_l: float = 0.154
    D_t: float = 0.0385
    gks_scale: float = 1.0
    gkr_scale: float = 1.0
    K_o: float = 5.4


@dataclass
class TissueCase:
    name: str
    xyz: np.ndarray
    tets: np.ndarray
    fibre: np.ndarray
    param_set: np.ndarray          # uint8 per cell
    stim_mask: np.ndarray          # uint8 per cell (bit k = protocol k)
    param_sets: list
    stimuli: list
    dt: float
    n_steps: int
    threshold: float
    output_steps: list = field(default_factory=list)
    tris: np.ndarray | None = None  # Purkinje-shell triangles (cells after the tets), or None

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_tris(self) -> int:
        return 0 if self.tris is None else int(self.tris.shape[0])

    @property
    def n_cells(self) -> int:
        return self.n_tets + self.n_tris

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])


def slab_case(nx=16, ny=16, nz=4, h=0.5, *, name="slab", dt=0.02,
              n_steps=1000, stim_x=1.0, threshold=-20.0, variant=0,
              D_l=0.154, D_t=0.0385, output_steps=(250, 500, 1000)) -> TissueCase:
    """Plain TP06 slab, fibres along x, zero-flux boundaries, stimulus
    -52 uA/uF for 1 ms in cells whose centroid has x < stim_x (mm).
    Defaults: 16x16x4 cubes of 0.5 mm = 6144 cells, 1000 steps of 0.02 ms."""
    xyz, tets = kuhn_box(nx, ny, nz, h)
    c = tet_centroids(xyz, tets)
    n = tets.shape[0]
    stim = (c[:, 0] < stim_x).astype(np.uint8)
    return TissueCase(name=name, xyz=xyz, tets=tets,
                      fibre=fibres_uniform(n), param_set=np.zeros(n, np.uint8),
                      stim_mask=stim,
                      param_sets=[ParamSet(model=0, variant=variant, D_l=D_l, D_t=D_t)],
                      stimuli=[Stimulus(-52.0, 0.0, 1.0)], dt=dt, n_steps=n_steps,
                      threshold=threshold, output_steps=list(output_steps))


def wedge_case(nx=200, ny=200, nz=40, h=0.25, *, name="wedge", dt=0.02,
               n_steps=20000, corner=1.5, threshold=-20.0,
               D_l=0.154, D_t=0.0385) -> TissueCase:
    """Ventricular wedge slab: fibre angle -60 deg (endo, z=0) to +60 deg (epi),
    TP06 endo/mid/epi variants in depth thirds, stimulus -52 uA/uF for 1 ms in
    the corner cube [0, corner]^3 mm. Defaults: 50x50x10 mm at 0.25 mm =
    9.6M cells."""
    xyz, tets = kuhn_box(nx, ny, nz, h)
    c = tet_centroids(xyz, tets)
    z_epi = nz * h
    fib = fibres_transmural(c[:, 2], 0.0, z_epi)
    third = z_epi / 3.0
    ps = np.where(c[:, 2] < third, PS_ENDO, np.where(c[:, 2] < 2 * third, PS_MID, PS_EPI)).astype(np.uint8)
    stim = np.all(c < corner, axis=1).astype(np.uint8)
    sets = [ParamSet(model=0, variant=0, D_l=D_l, D_t=D_t),
            ParamSet(model=0, variant=1, D_l=D_l, D_t=D_t),
            ParamSet(model=0, variant=2, D_l=D_l, D_t=D_t)]
    return TissueCase(name=name, xyz=xyz, tets=tets, fibre=fib, param_set=ps,
                      stim_mask=stim, param_sets=sets,
                      stimuli=[Stimulus(-52.0, 0.0, 1.0)], dt=dt, n_steps=n_steps,
                      threshold=threshold,
                      output_steps=list(range(250, n_steps + 1, 250)))


def sweep_jobs(n_jobs=256, n_min=50_000, n_max=2_000_000, h=0.25, seed_offset=4,
               scale=1.0):
    """Batched parametric sweep: slab jobs with log-uniform sizes, G_Ks/G_Kr
    scalings U[0.5,1.5], and with p=0.5 a spherical ischemic region (radius
    U[2,8] mm) where [K]o = 8 mM. Returns a list of dicts of job inputs
    (meshes built lazily by the caller through ``slab_from_spec``)."""
    rng = np.random.default_rng(MASTER_SEED + seed_offset)
    specs = []
    for j in range(n_jobs):
        target = math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale
        nz = max(1, int(round((target / (6 * 25)) ** (1.0 / 3.0))))
        nx = ny = 5 * nz
        gks, gkr = rng.uniform(0.5, 1.5, size=2)
        isch = rng.uniform() < 0.5
        radius = rng.uniform(2.0, 8.0)
        centre = rng.uniform(0.0, 1.0, size=3) * np.array([nx, ny, nz]) * h
        specs.append(dict(nx=nx, ny=ny, nz=nz, h=h, gks=float(gks), gkr=float(gkr),
                          ischemic=bool(isch), radius=float(radius),
                          centre=centre.tolist()))
    return specs


def slab_from_spec(spec, *, dt=0.02, n_steps=20000, threshold=-20.0) -> TissueCase:
    nx, ny, nz, h = spec["nx"], spec["ny"], spec["nz"], spec["h"]
    xyz, tets = kuhn_box(nx, ny, nz, h)
    c = tet_centroids(xyz, tets)
    n = tets.shape[0]
    ps = np.zeros(n, np.uint8)
    sets = [ParamSet(model=0, variant=0, gks_scale=spec["gks"], gkr_scale=spec["gkr"])]
    if spec["ischemic"]:
        inside = np.linalg.norm(c - np.asarray(spec["centre"]), axis=1) < spec["radius"]
        ps[inside] = 1
        sets.append(ParamSet(model=0, variant=0, gks_scale=spec["gks"],
                             gkr_scale=spec["gkr"], K_o=8.0))
    corner = min(1.5, nz * h)
    stim = np.all(c < corner, axis=1).astype(np.uint8)
    return TissueCase(name="sweep", xyz=xyz, tets=tets, fibre=fibres_uniform(n),
                      param_set=ps, stim_mask=stim, param_sets=sets,
                      stimuli=[Stimulus(-52.0, 0.0, 1.0)], dt=dt, n_steps=n_steps,
                      threshold=threshold)


def kuhn_cubes(mask: np.ndarray, h: float, origin=(0.0, 0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """Kuhn 6-tet split of the cubes where ``mask`` (shape nx, ny, nz) is
    True; cube (i, j, k) spans origin + h*[i, i+1] x ... . All cubes use the
    same split, so the mesh is conforming; only used nodes are kept."""
    nx, ny, nz = mask.shape
    ci, cj, ck = np.nonzero(mask)

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    tets = np.empty((ci.size, 6, 4), dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        pos = [ci.copy(), cj.copy(), ck.copy()]
        verts = [nid(*pos)]
        for ax in perm:
            pos[ax] = pos[ax] + 1
            verts.append(nid(*pos))
        parity = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b]) % 2
        if parity:
            verts[2], verts[3] = verts[3], verts[2]
        tets[:, t, :] = np.stack(verts, axis=1)
    tets = tets.reshape(-1, 4)
    used, inv = np.unique(tets, return_inverse=True)
    i = used % (nx + 1)
    j = (used // (nx + 1)) % (ny + 1)
    k = used // ((nx + 1) * (ny + 1))
    xyz = np.stack([i, j, k], axis=1).astype(np.float64) * h + np.asarray(origin, dtype=np.float64)
    return xyz, inv.reshape(-1, 4).astype(np.int32)


# Synthetic four-chamber topology (mm): two truncated ventricular ellipsoid
# shells (LV inside, RV wrapping its right side) below a base plane, and two
# atrial ellipsoid shells above it, electrically separate in 3D.
_LV_OUT, _LV_IN = (25.0, 25.0, 45.0), (17.0, 17.0, 37.0)
_RV_C, _RV_OUT, _RV_IN = (-14.0, 0.0, 0.0), (33.0, 26.0, 40.0), (28.0, 21.0, 35.0)
_BASE_Z = 20.0
_LA_C, _RA_C = (10.0, 0.0, 46.0), (-24.0, 0.0, 44.0)
_LA_OUT, _RA_OUT, _ATRIAL_WALL = (17.0, 16.0, 13.0), (18.0, 16.0, 13.0), 4.0


def _ell(p, c, ax):
    return np.sqrt(((p[..., 0] - c[0]) / ax[0]) ** 2 + ((p[..., 1] - c[1]) / ax[1]) ** 2
                   + ((p[..., 2] - c[2]) / ax[2]) ** 2)


def heart_regions(p):
    """Region label of points p (..., 3): 0 none, 1 LV, 2 RV, 3 LA, 4 RA, and
    the normalised transmural depth (0 endocardium, 1 epicardium)."""
    lv_o, lv_i = _ell(p, (0, 0, 0), _LV_OUT), _ell(p, (0, 0, 0), _LV_IN)
    rv_o, rv_i = _ell(p, _RV_C, _RV_OUT), _ell(p, _RV_C, _RV_IN)
    below = p[..., 2] < _BASE_Z
    lv = below & (lv_o <= 1.0) & (lv_i > 1.0)
    rv = below & (rv_o <= 1.0) & (rv_i > 1.0) & (lv_o > 1.0)
    la_o = _ell(p, _LA_C, _LA_OUT)
    la_i = _ell(p, _LA_C, tuple(a - _ATRIAL_WALL for a in _LA_OUT))
    ra_o = _ell(p, _RA_C, _RA_OUT)
    ra_i = _ell(p, _RA_C, tuple(a - _ATRIAL_WALL for a in _RA_OUT))
    la = (la_o <= 1.0) & (la_i > 1.0)
    ra = (ra_o <= 1.0) & (ra_i > 1.0) & ~la
    label = np.zeros(p.shape[:-1], np.uint8)
    label[lv], label[rv], label[la], label[ra] = 1, 2, 3, 4
    # depth from the inner to the outer surface along the ellipsoidal coordinate
    d = np.zeros(p.shape[:-1])
    d = np.where(lv, np.clip((lv_i - 1.0) / (lv_i - lv_o + 1e-9), 0, 1), d)
    d = np.where(rv, np.clip((rv_i - 1.0) / (rv_i - rv_o + 1e-9), 0, 1), d)
    d = np.where(la, np.clip((la_i - 1.0) / (la_i - la_o + 1e-9), 0, 1), d)
    d = np.where(ra, np.clip((ra_i - 1.0) / (ra_i - ra_o + 1e-9), 0, 1), d)
    return label, d


def heart_case(h: float = 0.4, *, scale: float = 1.0, dt: float = 0.02, n_steps: int = 40000,
               threshold: float = -20.0, av_delay: float = 100.0) -> TissueCase:
    """Synthetic whole-heart topology: ventricles (TP06, endo/epi variants by
    depth, fibres -60..+60 deg transmurally) and atria (Courtemanche,
    circumferential fibres) voxelised at spacing h and Kuhn-split; the
    geometry is scaled by ``scale``. Stimuli: a sinus-node sphere in the right
    atrium for 2.5 ms (Eq. 4), and, standing in for the conduction system, a
    sphere at the LV apex endocardium av_delay ms later."""
    lo = np.array([-50.0, -30.0, -47.0]) * scale
    hi = np.array([30.0, 30.0, 61.0]) * scale
    n = np.ceil((hi - lo) / h).astype(int)
    g = [lo[a] + h * (np.arange(n[a]) + 0.5) for a in range(3)]
    P = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1) / scale
    label, dep = heart_regions(P)
    mask = label > 0
    xyz, tets = kuhn_cubes(mask, h, lo)
    c = tet_centroids(xyz, tets) / scale
    # every tet takes the region and depth of its voxel (6 tets per voxel, in voxel order)
    lab = np.repeat(label[mask], 6)
    depth = np.repeat(dep[mask], 6)
    atrial = lab >= 3
    ps = np.where(atrial, 2, np.where(depth < 0.5, 1, 0)).astype(np.uint8)
    # fibres: circumferential around the chamber axis, rotated towards the long axis by alpha(depth)
    ctr = np.where((lab == 2)[:, None], np.array(_RV_C), 0.0)
    ctr = np.where((lab == 3)[:, None], np.array(_LA_C), ctr)
    ctr = np.where((lab == 4)[:, None], np.array(_RA_C), ctr)
    r = c - ctr
    t = np.stack([-r[:, 1], r[:, 0], np.zeros(len(r))], axis=1)
    t /= np.maximum(np.linalg.norm(t, axis=1, keepdims=True), 1e-9)
    alpha = np.where(atrial, 0.0, np.deg2rad(-60.0 + 120.0 * depth))
    fib = np.cos(alpha)[:, None] * t + np.sin(alpha)[:, None] * np.array([0.0, 0.0, 1.0])
    sinus = np.linalg.norm(c - (np.array(_RA_C) + [0, 0, 11.0]), axis=1) < 3.0
    apex = np.linalg.norm(c - np.array([0.0, 0.0, -38.0]), axis=1) < 4.0
    smask = (sinus.astype(np.uint8) | (apex.astype(np.uint8) << 1))
    sets = [ParamSet(model=0, variant=0), ParamSet(model=0, variant=2),
            ParamSet(model=1, D_l=0.154 * 1.05, D_t=0.0385 * 1.05)]
    return TissueCase(name="heart", xyz=xyz, tets=tets, fibre=fib, param_set=ps, stim_mask=smask,
                      param_sets=sets, stimuli=[Stimulus(-52.0, 0.0, 2.5), Stimulus(-52.0, av_delay, 2.0)],
                      dt=dt, n_steps=n_steps, threshold=threshold)


def heart_h_for_cells(target_cells: int, scale: float = 1.0) -> float:
    """Voxel spacing giving about target_cells tets for heart_case at this scale
    (tissue volume measured once on a coarse grid)."""
    hc = 1.0
    lo = np.array([-50.0, -30.0, -47.0])
    hi = np.array([30.0, 30.0, 61.0])
    n = np.ceil((hi - lo) / hc).astype(int)
    g = [lo[a] + hc * (np.arange(n[a]) + 0.5) for a in range(3)]
    P = np.stack(np.meshgrid(*g, indexing="ij"), axis=-1)
    vol = float((heart_regions(P)[0] > 0).sum()) * hc ** 3 * scale ** 3
    return (6.0 * vol / max(target_cells, 1)) ** (1.0 / 3.0)


@dataclass
class GraphParams:
    """Coupling parameters of a conduction graph (units mm, ms, mV, uA/uF)."""
    D: float = 2.82                 # Purkinje: 3.95 mS/mm / (chi C_m) (Table 2)
    g_graph: float = 0.5            # resistive junction rates, 1/ms
    g_cell: float = 0.05
    threshold: float = 0.0          # triggered: V crossing threshold (Sec. 3.3: 0 mV)
    delay_ortho: float = 5.0        # Purkinje -> muscle delay (Sec. 3.3)
    delay_anti: float = 3.0         # muscle -> Purkinje delay (Sec. 1: 2-3 ms)
    amplitude: float = -52.0
    duration: float = 0.5           # S_d of a communication-node stimulus (Sec. 3.3)
    radius: float = 0.1             # R_S (Sec. 3.3: 0.1 mm Purkinje, 1 mm atria)
    two_way: int = 0
    substeps: int = 0               # 0 = chosen from the stability bound


JUNC_RESISTIVE, JUNC_TRIGGERED, JUNC_CELL = 0, 1, 2   # JUNC_CELL: junction_node is a source cell


@dataclass
class Graph:
    xyz: np.ndarray
    edges: np.ndarray
    param_set: np.ndarray
    stim_mask: np.ndarray
    junction_node: np.ndarray
    junction_cell: np.ndarray
    junction_mode: np.ndarray
    params: GraphParams
    edge_D: np.ndarray | None = None

    @property
    def n_nodes(self):
        return int(self.xyz.shape[0])


def chain_graph(n, ds, start=(0.0, 0.0, 0.0), direction=(1.0, 0.0, 0.0), *, param_set=0, stim_nodes=0,
                params=None):
    """A straight cable of n nodes spaced ds mm; the first stim_nodes nodes
    carry stimulus protocol 0."""
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    xyz = np.asarray(start, float) + ds * np.arange(n)[:, None] * d
    edges = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int32)
    sm = np.zeros(n, np.uint8)
    sm[:stim_nodes] = 1
    return Graph(xyz, edges, np.full(n, param_set, np.uint8), sm, np.zeros(0, np.int32), np.zeros(0, np.int32),
                 np.zeros(0, np.uint8), params or GraphParams())


def _project(q, c, ax):
    """Radial projection of q onto the ellipsoid (centre c, semi-axes ax)."""
    r = _ell(q[None], c, ax)[0]
    return np.asarray(c) + (q - np.asarray(c)) / r


def _normal(q, c, ax):
    g = 2.0 * (q - np.asarray(c)) / np.asarray(ax) ** 2
    return g / np.linalg.norm(g)


def _rotate(v, axis, th):
    """Rodrigues rotation of v about a unit axis by th radians."""
    return (v * np.cos(th) + np.cross(axis, v) * np.sin(th) + axis * np.dot(axis, v) * (1 - np.cos(th)))


def grow_tree(rng, start, centre, axes, n_target, ds=0.2, seg_len=(1.0, 3.0), angle_deg=(30.0, 60.0),
              z_max=18.0, first_dir=(0.0, 0.0, -1.0)):
    """Seeded fractal tree on an ellipsoidal surface: straight segments of
    length U[seg_len] sampled every ds, each ending in a bifurcation whose
    children turn by +/- U[angle_deg] about the surface normal; nodes are
    projected onto the surface; branches stop above z_max (the base).
    Returns (xyz, edges, parent-order node list); node 0 is `start`."""
    start = _project(np.asarray(start, float), centre, axes)
    xyz, edges = [start], []
    d0 = np.asarray(first_dir, float)
    n0 = _normal(start, centre, axes)
    d0 = d0 - np.dot(d0, n0) * n0
    active = [(0, d0 / np.linalg.norm(d0))]
    while active and len(xyz) < n_target:
        i, d = active.pop(0)
        p, prev = xyz[i], i
        m = max(1, int(round(rng.uniform(*seg_len) / ds)))
        ok = True
        for _ in range(m):
            q = _project(p + ds * d, centre, axes)
            if q[2] > z_max:
                ok = False
                break
            xyz.append(q)
            edges.append((prev, len(xyz) - 1))
            d = (q - p) / np.linalg.norm(q - p)
            p, prev = q, len(xyz) - 1
            if len(xyz) >= n_target:
                break
        if not ok or prev == i:
            continue
        nrm = _normal(p, centre, axes)
        for sign in (1.0, -1.0):
            th = np.deg2rad(rng.uniform(*angle_deg))
            d2 = _rotate(d, nrm, sign * th)
            d2 -= np.dot(d2, nrm) * nrm
            active.append((prev, d2 / np.linalg.norm(d2)))
    return np.array(xyz), np.array(edges, np.int32).reshape(-1, 2)


def whole_heart(h: float = 0.4, *, scale: float = 1.0, n_tree: int = 50_000, n_pmj: int = 2000,
                ds: float = 0.2, dt: float = 0.02, n_steps: int = 40_000, seed: int = 3,
                g_graph: float = 0.3, g_cell: float = 4.0):
    """Synthetic whole-heart topology with its conduction system:
    ventricles (TP06) and atria (Courtemanche) from heart_case; an atrial
    bundle (Courtemanche, Table 2 1D conductivity) from the sinus node over
    the right atrium to the AV node, with a branch to the left atrium; a low
    diffusivity AV delay line to the His root; and two seeded fractal Stewart
    trees (left and right bundle branches, Table 2 Purkinje conductivity)
    grown on the ventricular endocardia until n_tree nodes in all. Up to
    n_pmj tree terminals are paired with their nearest ventricular cell
    through resistive junctions (PMJs); every 5th bundle node is a
    communication node that triggers the nearest atrial cells (R_S = 1 mm,
    Sec. 3.3). A sinus stimulus (S_d = 2.5 ms, Eq. 4) excites the sinus
    node in 3D and the first bundle nodes. Geometry scaled by `scale`.
    Returns (TissueCase, Graph)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(MASTER_SEED + 3 + seed)
    case = heart_case(h=h, scale=scale, dt=dt, n_steps=n_steps, av_delay=1e9)
    case.param_sets.append(ParamSet(model=2))                 # set 3: Stewart (Purkinje)
    ds_s = ds / scale                                          # node spacing in unscaled units
    # atrial bundle over the right-atrial endocardium, sinus node -> AV node, with a branch to the LA
    ra_ax = tuple(a - _ATRIAL_WALL + 0.5 for a in _RA_OUT)
    la_ax = tuple(a - _ATRIAL_WALL + 0.5 for a in _LA_OUT)
    sinus = np.array(_RA_C) + [0.0, 0.0, 11.0]
    avn = np.array(_RA_C) + [12.0, 0.0, -9.0]

    def surface_path(a, b, c, ax):
        # project a dense chord onto the surface, then resample at equal arc length ds
        dense = np.array([_project(a + (b - a) * t, c, ax) for t in np.linspace(0, 1, 2001)])
        s_arc = np.concatenate([[0.0], np.cumsum(np.linalg.norm(np.diff(dense, axis=0), axis=1))])
        m = max(2, int(np.ceil(s_arc[-1] / ds_s)))
        t = np.linspace(0, s_arc[-1], m + 1)
        return np.stack([np.interp(t, s_arc, dense[:, k]) for k in range(3)], axis=1)
    ra_path = surface_path(sinus, avn, _RA_C, ra_ax)
    mid = ra_path[len(ra_path) // 3]
    bach = surface_path(mid, np.array(_LA_C) + [-6.0, 0.0, 8.0], _LA_C, la_ax)
    his = np.array([-8.0, 0.0, 17.0])
    av_line = np.array([avn + (his - avn) * t
                        for t in np.linspace(0, 1, int(np.ceil(np.linalg.norm(his - avn) / ds_s)) + 1)])
    xyz = [ra_path, bach[1:], av_line[1:]]
    edges = [np.stack([np.arange(len(ra_path) - 1), np.arange(1, len(ra_path))], 1)]
    o = len(ra_path)
    imid = len(ra_path) // 3
    eb = [(imid, o)] + [(o + k, o + k + 1) for k in range(len(bach) - 2)]
    edges.append(np.array(eb))
    o2 = o + len(bach) - 1
    ea = [(len(ra_path) - 1, o2)] + [(o2 + k, o2 + k + 1) for k in range(len(av_line) - 2)]
    edges.append(np.array(ea))
    n_bundle = o2                                             # bundle nodes (Courtemanche, fast)
    av_end = o2 + len(av_line) - 2
    # the AV delay line's diffusivity slows conduction to about 0.18 mm/ms, i.e. ~100 ms over
    # its 18 mm at full scale (delays shrink with the geometry when scale < 1)
    D_bundle, D_av, D_purk = 1.29 / 1.4, 0.038, 3.95 / 1.4
    edge_D = [np.full(len(ra_path) - 1, D_bundle), np.full(len(eb), D_bundle), np.full(len(ea), D_av)]
    # His bundle: a short Stewart segment whose diffusivity rises geometrically from the AV line's
    # to the Purkinje value, so that the slow line can drive the two fast branches
    n_his = 15
    his_seg = np.array([his + [0.0, 0.0, -ds_s * (k + 1)] for k in range(n_his)])
    xyz.append(his_seg)
    o3 = av_end + 1
    edges.append(np.array([(av_end, o3)] + [(o3 + k, o3 + k + 1) for k in range(n_his - 1)]))
    edge_D.append(D_av * (D_purk / D_av) ** (np.arange(1, n_his + 1) / n_his))
    his_idx = o3 + n_his - 1
    his = his_seg[-1]
    # left and right bundle branches on the endocardia
    base = his_idx + 1
    node_off = base
    tree_nodes = []
    lv_ax = tuple(a + 0.6 for a in _LV_IN)
    rv_ax = tuple(a + 0.6 for a in _RV_IN)
    # each branch starts on its chamber's septal endocardium below the base and grows downwards
    n_edges_before = sum(len(e) for e in edges)
    branch_edges = []
    for c, ax, share, sdir in (((0.0, 0.0, 0.0), lv_ax, 0.55, (-1.0, 0.0, 0.35)),
                               (_RV_C, rv_ax, 0.45, (1.0, 0.0, 0.35))):
        start = np.asarray(c) + 10.0 * np.asarray(sdir)
        txyz, tedges = grow_tree(rng, start, c, ax, int(n_tree * share), ds=ds_s, z_max=_BASE_Z - 2.0)
        xyz.append(txyz)
        edges.append(tedges + node_off)
        edges.append(np.array([[his_idx, node_off]]))
        edge_D += [np.full(len(tedges), D_purk), np.array([D_purk])]
        tree_nodes.append((node_off, len(txyz), tedges))
        branch_edges.append(np.arange(n_edges_before, n_edges_before + len(tedges) + 1))
        n_edges_before += len(tedges) + 1
        node_off += len(txyz)
    gxyz = np.concatenate(xyz) * scale
    gedges = np.concatenate(edges).astype(np.int32)
    gD = np.concatenate(edge_D)
    n = gxyz.shape[0]
    pset = np.full(n, 3, np.uint8)
    pset[:av_end + 1] = 2                                     # bundle and AV line: Courtemanche
    smask = np.zeros(n, np.uint8)
    smask[:max(5, int(round(2.0 / ds)))] = 1                  # sinus stimulus on the first 2 mm of bundle
    cen = tet_centroids(case.xyz, case.tets)
    vent = case.param_set <= 1
    atr = case.param_set == 2
    kv = cKDTree(cen[vent])
    ka = cKDTree(cen[atr])
    vid, aid = np.flatnonzero(vent), np.flatnonzero(atr)
    deg = np.bincount(gedges.ravel(), minlength=n)
    leaves = np.array([i for i in range(base, n) if deg[i] == 1])
    if len(leaves) > n_pmj:
        leaves = leaves[np.linspace(0, len(leaves) - 1, n_pmj).astype(int)]
    _, pm = kv.query(gxyz[leaves])
    cn = np.arange(0, n_bundle, 5)
    _, ac = ka.query(gxyz[cn])
    jn = np.concatenate([leaves, cn]).astype(np.int32)
    jc = np.concatenate([vid[pm], aid[ac]]).astype(np.int32)
    jm = np.concatenate([np.full(len(leaves), JUNC_RESISTIVE), np.full(len(cn), JUNC_TRIGGERED)]).astype(np.uint8)
    gp = GraphParams(D=D_purk, g_graph=g_graph, g_cell=g_cell, threshold=0.0, delay_ortho=5.0, delay_anti=3.0,
                     amplitude=-52.0, duration=0.5, radius=1.0 * scale)
    case.stimuli[0] = Stimulus(-100.0, 0.0, 2.5)
    graph = Graph(gxyz, gedges, pset, smask, jn, jc, jm, gp, edge_D=gD)
    graph.n_bundle, graph.his = n_bundle, his_idx
    # edge and node sets of the parts, for pathology scenarios (heart_scenario)
    graph.av_edges = np.arange(len(ra_path) - 1 + len(eb), len(ra_path) - 1 + len(eb) + len(ea))
    graph.lv_edges, graph.rv_edges = branch_edges
    graph.lv_nodes = np.arange(tree_nodes[0][0], tree_nodes[0][0] + tree_nodes[0][1])
    graph.rv_nodes = np.arange(tree_nodes[1][0], tree_nodes[1][0] + tree_nodes[1][1])
    graph.scale = scale
    return case, graph


def heart_lead_site(case: TissueCase, graph: Graph, site: str) -> np.ndarray:
    """Lead sites of Sec. 5 on the synthetic heart (case coordinates): the
    right-ventricular apex ("rv_apex": the lowest right-ventricular cell) or
    the right-atrial appendage ("ra_appendage": the most lateral right-atrial
    cell)."""
    cen = tet_centroids(case.xyz, case.tets)
    lab, _ = heart_regions(cen / graph.scale)
    if site == "rv_apex":
        k = np.flatnonzero(lab == 2)
        return cen[k[np.argmin(cen[k, 2])]]
    if site == "ra_appendage":
        k = np.flatnonzero(lab == 4)
        return cen[k[np.argmin(cen[k, 0])]]
    raise ValueError(site)


def heart_scenario(case: TissueCase, graph: Graph, *, block: str | None = None, severity: float = 1.0,
                   av_block: bool = False, sinus: bool = True, lead=None, lead_radius: float = 2.0,
                   lead_onset: float = 0.0, lead_period: float = 0.0, lead_amp: float = -100.0,
                   lead_dur: float = 2.0, two_way: bool | None = None, cn_amplitude: float | None = None,
                   cn_duration: float | None = None):
    """Pathology and pacing variants of a whole-heart case (Sec. 5), as inputs only:
    - block "left" / "right": bundle-branch block, the branch's conductivity
      scaled by (1 - severity) (severity 1: null conductivity, complete block);
    - av_block: null conductivity along the AV delay line;
    - sinus False: no sinus-node stimulus;
    - two_way: the communication nodes also let the myocardium excite the
      graph (Sec. 3.3: pathological cases), else as built; cn_amplitude /
      cn_duration replace the communication-node stimulus (a single 1D node
      is tightly coupled to its cable neighbours, so exciting it takes a
      larger current than exciting a patch of myocardium);
    - lead (a site name of heart_lead_site or a point): a pacing lead, a
      stimulus protocol (lead_amp uA/uF for lead_dur ms from lead_onset,
      every lead_period ms; 0 = once) on the myocardial cells within
      lead_radius mm of the point.
    Returns new (case, graph); the inputs are not modified."""
    import copy
    c2, g2 = copy.deepcopy(case), copy.deepcopy(graph)
    D = np.array(g2.edge_D, dtype=np.float64)
    if block is not None:
        D[g2.lv_edges if block == "left" else g2.rv_edges] *= (1.0 - severity)
    if av_block:
        D[g2.av_edges] = 0.0
    g2.edge_D = D
    if two_way is not None:
        g2.params = replace(g2.params, two_way=int(two_way))
    if cn_amplitude is not None:
        g2.params = replace(g2.params, amplitude=float(cn_amplitude))
    if cn_duration is not None:
        g2.params = replace(g2.params, duration=float(cn_duration))
    if not sinus:   # protocol 0 drives the sinus node: the first bundle nodes and the RA sphere
        g2.stim_mask = np.zeros_like(g2.stim_mask)
        c2.stim_mask = c2.stim_mask & np.uint8(0xFE)
    if lead is not None:
        cen = tet_centroids(c2.xyz, c2.tets)
        p = heart_lead_site(c2, g2, lead) if isinstance(lead, str) else np.asarray(lead, float)
        d = np.linalg.norm(cen - p, axis=1)
        sel = d <= lead_radius
        k = len(c2.stimuli)
        c2.stimuli = list(c2.stimuli) + [Stimulus(lead_amp, lead_onset, lead_dur, lead_period)]
        c2.stim_mask = c2.stim_mask | (sel.astype(np.uint8) << k)
    return c2, g2
