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
from dataclasses import dataclass, field

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

    @property
    def n_cells(self) -> int:
        return int(self.tets.shape[0])

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


JUNC_RESISTIVE, JUNC_TRIGGERED = 0, 1


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
