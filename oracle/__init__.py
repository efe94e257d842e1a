"""FP64 CPU oracle for the monodomain finite-volume step.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it to check and time the CUDA library; the product never
imports it. It is plain C (``*.c`` in this folder) following the paper's
algorithm stage by stage (see ``oracle.h``), compiled with gcc into
``liboracle.so``; this module only marshals arguments through ctypes.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
  - geometry, S1-S3 diffusion operator: pinned (conservation, row sums,
    linear patch test, cosine-eigenmode decay and its O(h^2) convergence,
    fibre-rotation decay rates, two-point symmetry, hand-derived two-tet case);
  - TP06 / Courtemanche / Stewart: physiological pins (rest potential, APD,
    plateau, RL closed form, first-order time convergence) and the charge
    balance between the V equation and the ion concentrations (exact for
    TP06 and Stewart, exact up to the stimulus charge and a first-order
    buffering error for Courtemanche). Parity with the published model
    traces is unpinned: the model papers' figures and reference code are not
    available here;
  - the conduction graph, the 2D shell, the bidomain solve and AB2: pinned in
    their own test files (conservation, closed forms, convergence orders,
    reductions to the monodomain case).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
SOURCES = ["fv3d.c", "fv2d.c", "tp06.c", "crn.c", "stewart.c", "tissue.c", "purkinje.c"]

TP06, CRN, STEWART = 0, 1, 2
MAXVAR = 24


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, IEEE semantics, OpenMP over cells)."""
    srcs = [os.path.join(_HERE, s) for s in SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr, __file__])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class CellParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("D_l", ctypes.c_double), ("D_t", ctypes.c_double),
                ("gks_scale", ctypes.c_double), ("gkr_scale", ctypes.c_double),
                ("K_o", ctypes.c_double)]


class GraphParams(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("g_graph", ctypes.c_double), ("g_cell", ctypes.c_double),
                ("threshold", ctypes.c_double), ("delay_ortho", ctypes.c_double),
                ("delay_anti", ctypes.c_double), ("amplitude", ctypes.c_double), ("duration", ctypes.c_double),
                ("radius", ctypes.c_double), ("two_way", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("act_threshold", ctypes.c_double)]


class Stim(ctypes.Structure):
    _fields_ = [("amplitude", ctypes.c_double), ("t_on", ctypes.c_double),
                ("duration", ctypes.c_double), ("period", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_mesh_create.restype = _P
        L.orc_mesh_create.argtypes = [ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_int)]
        L.orc_mesh_destroy.argtypes = [_P]
        L.orc_mesh_n_boundary_faces.restype = ctypes.c_int64
        L.orc_mesh_n_boundary_faces.argtypes = [_P]
        L.orc_mesh_cell_info.argtypes = [_P, _P, _P, _P]
        for f in ("orc_node_values", "orc_cell_gradients"):
            getattr(L, f).argtypes = [_P, _P, _P]
        for f in ("orc_diffusion", "orc_diffusion_twopoint"):
            getattr(L, f).argtypes = [_P, _P, _P, _P]
        L.orc_conductivity.argtypes = [_P, ctypes.c_double, ctypes.c_double, _P]
        L.orc_model_nvar.restype = ctypes.c_int
        L.orc_model_nvar.argtypes = [ctypes.c_int]
        L.orc_model_varname.restype = ctypes.c_char_p
        L.orc_model_varname.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_model_init.argtypes = [ctypes.POINTER(CellParams), _P]
        L.orc_model_step.restype = ctypes.c_double
        L.orc_model_step.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(CellParams), _P]
        L.orc_sim_set_integrator.restype = ctypes.c_int
        L.orc_sim_set_integrator.argtypes = [_P, ctypes.c_int]
        L.orc_cell_run.argtypes = [ctypes.POINTER(CellParams), ctypes.c_double, ctypes.c_int64,
                                   ctypes.POINTER(Stim), ctypes.c_int64, _P, _P, ctypes.c_int]
        L.orc_sim_create.restype = _P
        L.orc_sim_create.argtypes = [ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P, _P,
                                     ctypes.c_int, _P, ctypes.c_int, _P,
                                     ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        L.orc_sim_create2.restype = _P
        L.orc_sim_create2.argtypes = [ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P, _P,
                                      ctypes.c_int, _P, ctypes.c_int, _P,
                                      ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        L.orc_shell_create.restype = _P
        L.orc_shell_create.argtypes = [ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_int)]
        L.orc_shell_destroy.argtypes = [_P]
        L.orc_shell_node_values.argtypes = [_P, _P, _P]
        L.orc_shell_gradients.argtypes = [_P, _P, _P]
        L.orc_shell_diffusion.argtypes = [_P, _P, _P, _P]
        L.orc_shell_cell_info.argtypes = [_P, _P, _P, _P]
        L.orc_sim_destroy.argtypes = [_P]
        L.orc_sim_run.argtypes = [_P, ctypes.c_int64]
        L.orc_sim_step_index.restype = ctypes.c_int64
        L.orc_sim_step_index.argtypes = [_P]
        L.orc_sim_set_step_index.argtypes = [_P, ctypes.c_int64]
        L.orc_sim_get_var.argtypes = [_P, ctypes.c_int, _P]
        L.orc_sim_set_var.argtypes = [_P, ctypes.c_int, _P]
        L.orc_sim_get_act.argtypes = [_P, _P]
        L.orc_sim_diffusion.argtypes = [_P, _P, _P]
        L.orc_sim_attach_graph.restype = ctypes.c_int
        L.orc_sim_attach_graph.argtypes = [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P, _P,
                                           ctypes.c_int64, _P, _P, _P, ctypes.POINTER(GraphParams)]
        L.orc_sim_graph_substeps.restype = ctypes.c_int
        L.orc_sim_graph_substeps.argtypes = [_P]
        for f in ("orc_sim_graph_get_var", "orc_sim_graph_set_var"):
            getattr(L, f).argtypes = [_P, ctypes.c_int, _P]
        L.orc_sim_graph_get_act.argtypes = [_P, _P]
        L.orc_sim_graph_laplacian.argtypes = [_P, _P, _P]
        L.orc_stim_active.restype = ctypes.c_int
        L.orc_sim_set_bidomain.restype = ctypes.c_int
        L.orc_sim_set_bidomain.argtypes = [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int64]
        for f in ("orc_sim_get_ve", "orc_sim_set_ve", "orc_sim_bidomain_stats"):
            getattr(L, f).argtypes = [_P, _P]
        L.orc_sim_bidomain_operator.argtypes = [_P, _P, _P]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_stim_active.argtypes = [ctypes.POINTER(Stim), ctypes.c_double, ctypes.c_int64]
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Thread count of the oracle's OpenMP loops for later calls from this
    thread (n <= 0 leaves it); returns the previous count."""
    return int(lib().orc_set_threads(int(n)))


def conductivity(fibre, D_l, D_t) -> np.ndarray:
    f = np.ascontiguousarray(fibre, dtype=np.float64)
    D = np.zeros(9)
    lib().orc_conductivity(_ptr(f), float(D_l), float(D_t), _ptr(D))
    return D.reshape(3, 3)


class Mesh:
    """Oracle geometry of a tetrahedral mesh and its diffusion operator."""

    def __init__(self, xyz, tets):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        err = ctypes.c_int(0)
        self._h = lib().orc_mesh_create(self.xyz.shape[0], _ptr(self.xyz), self.tets.shape[0],
                                         _ptr(self.tets), ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle mesh rejected (code {err.value})")
        self.n_cells = self.tets.shape[0]
        self.n_nodes = self.xyz.shape[0]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_mesh_destroy(self._h)
            self._h = None

    @property
    def n_boundary_faces(self):
        return int(lib().orc_mesh_n_boundary_faces(self._h))

    def cell_info(self):
        c = np.zeros((self.n_cells, 3))
        v = np.zeros(self.n_cells)
        nb = np.zeros((self.n_cells, 4), np.int32)
        lib().orc_mesh_cell_info(self._h, _ptr(c), _ptr(v), _ptr(nb))
        return c, v, nb

    def node_values(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n_nodes)
        lib().orc_node_values(self._h, _ptr(v), _ptr(out))
        return out

    def cell_gradients(self, vn):
        vn = np.ascontiguousarray(vn, dtype=np.float64)
        out = np.zeros((self.n_cells, 3))
        lib().orc_cell_gradients(self._h, _ptr(vn), _ptr(out))
        return out

    def tensors(self, fibre, D_l, D_t):
        fibre = np.asarray(fibre, dtype=np.float64).reshape(-1, 3)
        D_l = np.broadcast_to(np.asarray(D_l, dtype=np.float64), (self.n_cells,))
        D_t = np.broadcast_to(np.asarray(D_t, dtype=np.float64), (self.n_cells,))
        return np.stack([conductivity(fibre[c], D_l[c], D_t[c]) for c in range(self.n_cells)])

    def diffusion(self, D, v, twopoint=False):
        D = np.ascontiguousarray(D, dtype=np.float64).reshape(self.n_cells, 9)
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n_cells)
        f = lib().orc_diffusion_twopoint if twopoint else lib().orc_diffusion
        f(self._h, _ptr(D), _ptr(v), _ptr(out))
        return out


class Shell:
    """Oracle geometry of a triangle surface (the Purkinje shell) and its
    diffusion operator (see ``fv2d.c``)."""

    def __init__(self, xyz, tris):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        err = ctypes.c_int(0)
        self._h = lib().orc_shell_create(self.xyz.shape[0], _ptr(self.xyz), self.tris.shape[0], _ptr(self.tris),
                                         ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle shell rejected (code {err.value})")
        self.n_cells = self.tris.shape[0]
        self.n_nodes = self.xyz.shape[0]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_shell_destroy(self._h)
            self._h = None

    def cell_info(self):
        c = np.zeros((self.n_cells, 3))
        a = np.zeros(self.n_cells)
        nb = np.zeros((self.n_cells, 3), np.int32)
        lib().orc_shell_cell_info(self._h, _ptr(c), _ptr(a), _ptr(nb))
        return c, a, nb

    def node_values(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n_nodes)
        lib().orc_shell_node_values(self._h, _ptr(v), _ptr(out))
        return out

    def cell_gradients(self, vn):
        vn = np.ascontiguousarray(vn, dtype=np.float64)
        out = np.zeros((self.n_cells, 3))
        lib().orc_shell_gradients(self._h, _ptr(vn), _ptr(out))
        return out

    def diffusion(self, D, v):
        D = np.ascontiguousarray(np.broadcast_to(np.asarray(D, np.float64).reshape(-1, 9), (self.n_cells, 9)))
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n_cells)
        lib().orc_shell_diffusion(self._h, _ptr(D), _ptr(v), _ptr(out))
        return out


def model_nvar(model: int) -> int:
    return int(lib().orc_model_nvar(model))


def model_varnames(model: int) -> list[str]:
    return [lib().orc_model_varname(model, k).decode() for k in range(model_nvar(model))]


def _cellparams(p) -> CellParams:
    if isinstance(p, CellParams):
        return p
    return CellParams(int(p.model), int(p.variant), float(p.D_l), float(p.D_t),
                      float(p.gks_scale), float(p.gkr_scale), float(p.K_o))


def _stim(s) -> Stim:
    if s is None or isinstance(s, Stim):
        return s
    return Stim(float(s.amplitude), float(s.t_on), float(s.duration), float(s.period))


def model_init(params) -> np.ndarray:
    s = np.zeros(MAXVAR)
    lib().orc_model_init(ctypes.byref(_cellparams(params)), _ptr(s))
    return s


def model_step(state, dt, i_stim, params) -> float:
    """One RL/FE update of every variable but V; returns I_ion(V^n, s^n)."""
    assert state.dtype == np.float64 and state.size >= MAXVAR
    return float(lib().orc_model_step(_ptr(state), float(dt), float(i_stim),
                                      ctypes.byref(_cellparams(params)), None))


def cell_run(params, dt, n_steps, stim=None, record_every=1, state=None, integrator=0):
    """Single-cell run; returns (V every record_every steps, final state).
    integrator 1: AB2 for the non-gating variables."""
    st = model_init(params) if state is None else np.array(state, dtype=np.float64)
    nrec = n_steps // record_every if record_every > 0 else 0
    v = np.zeros(max(nrec, 1))
    sp = _stim(stim)
    lib().orc_cell_run(ctypes.byref(_cellparams(params)), float(dt), int(n_steps),
                       ctypes.byref(sp) if sp is not None else None, int(record_every),
                       _ptr(v), _ptr(st), int(integrator))
    return v[:nrec], st


def stim_active(stim, dt, n) -> bool:
    return bool(lib().orc_stim_active(ctypes.byref(_stim(stim)), float(dt), int(n)))


class Sim:
    """Oracle tissue simulation of one job (see ``tissue.c``)."""

    def __init__(self, case):
        self.case = case
        self.xyz = np.ascontiguousarray(case.xyz, dtype=np.float64)
        self.tets = np.ascontiguousarray(case.tets, dtype=np.int32)
        self.fibre = np.ascontiguousarray(case.fibre, dtype=np.float64)
        self.pset = np.ascontiguousarray(case.param_set, dtype=np.uint8)
        self.smask = np.ascontiguousarray(case.stim_mask, dtype=np.uint8)
        self.sets = (CellParams * len(case.param_sets))(*[_cellparams(p) for p in case.param_sets])
        ns = len(case.stimuli)
        self.stims = (Stim * max(ns, 1))(*[_stim(s) for s in case.stimuli])
        err = ctypes.c_int(0)
        tris = getattr(case, "tris", None)
        self.tris = np.ascontiguousarray(tris if tris is not None else np.zeros((0, 3)), dtype=np.int32)
        self._h = lib().orc_sim_create2(self.xyz.shape[0], _ptr(self.xyz), self.tets.shape[0],
                                        _ptr(self.tets), self.tris.shape[0], _ptr(self.tris), _ptr(self.fibre),
                                        _ptr(self.pset), _ptr(self.smask), len(case.param_sets),
                                        ctypes.cast(self.sets, _P), ns, ctypes.cast(self.stims, _P),
                                        float(case.dt), float(case.threshold), ctypes.byref(err))
        if not self._h:
            raise ValueError(f"oracle simulation rejected (code {err.value})")
        self.n_cells = self.tets.shape[0] + self.tris.shape[0]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_sim_destroy(self._h)
            self._h = None

    def run(self, n_steps):
        lib().orc_sim_run(self._h, int(n_steps))

    def set_integrator(self, integrator: int) -> None:
        """0 forward Euler, 1 AB2 for the non-gating variables (from now on)."""
        if lib().orc_sim_set_integrator(self._h, int(integrator)):
            raise ValueError("unknown integrator")

    @property
    def step_index(self) -> int:
        return int(lib().orc_sim_step_index(self._h))

    @step_index.setter
    def step_index(self, n):
        lib().orc_sim_set_step_index(self._h, int(n))

    def get(self, var: int) -> np.ndarray:
        out = np.zeros(self.n_cells)
        lib().orc_sim_get_var(self._h, int(var), _ptr(out))
        return out

    def set(self, var: int, values) -> None:
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.size == self.n_cells
        lib().orc_sim_set_var(self._h, int(var), _ptr(v))

    @property
    def V(self) -> np.ndarray:
        return self.get(0)

    def activation_times(self) -> np.ndarray:
        out = np.zeros(self.n_cells)
        lib().orc_sim_get_act(self._h, _ptr(out))
        return out

    def set_bidomain(self, De_l, De_t, tol=1e-10, restart=20, max_iter=200000):
        """Bidomain model: the parameter sets' (D_l, D_t) become the
        intracellular diffusivities; De_l, De_t (scalars or one per set) the
        extracellular ones. v_e is solved at once from the current V."""
        k = len(self.case.param_sets)
        el = np.ascontiguousarray(np.broadcast_to(np.asarray(De_l, np.float64), (k,)))
        et = np.ascontiguousarray(np.broadcast_to(np.asarray(De_t, np.float64), (k,)))
        rc = lib().orc_sim_set_bidomain(self._h, _ptr(el), _ptr(et), float(tol), int(restart), int(max_iter))
        if rc:
            raise ValueError(f"oracle bidomain rejected (code {rc})")

    @property
    def ve(self) -> np.ndarray:
        out = np.zeros(self.n_cells)
        lib().orc_sim_get_ve(self._h, _ptr(out))
        return out

    @ve.setter
    def ve(self, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.size == self.n_cells
        lib().orc_sim_set_ve(self._h, _ptr(v))

    def bidomain_stats(self) -> dict:
        st = np.zeros(4)
        lib().orc_sim_bidomain_stats(self._h, _ptr(st))
        return {"last_iters": int(st[0]), "total_iters": int(st[1]), "last_rel_res": float(st[2]),
                "failed": bool(st[3])}

    def bidomain_operator(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(self.n_cells)
        lib().orc_sim_bidomain_operator(self._h, _ptr(x), _ptr(out))
        return out

    def diffusion(self, v) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n_cells)
        lib().orc_sim_diffusion(self._h, _ptr(v), _ptr(out))
        return out

    def attach_graph(self, graph):
        """graph: an object with xyz, edges, edge_D (or None), param_set,
        stim_mask, junction_node, junction_cell, junction_mode and params
        (fields of GraphParams)."""
        keep = [np.ascontiguousarray(graph.xyz, dtype=np.float64),
                np.ascontiguousarray(graph.edges, dtype=np.int32),
                None if graph.edge_D is None else np.ascontiguousarray(graph.edge_D, dtype=np.float64),
                np.ascontiguousarray(graph.param_set, dtype=np.uint8),
                np.ascontiguousarray(graph.stim_mask, dtype=np.uint8),
                np.ascontiguousarray(graph.junction_node, dtype=np.int32),
                np.ascontiguousarray(graph.junction_cell, dtype=np.int32),
                np.ascontiguousarray(graph.junction_mode, dtype=np.uint8)]
        gp = graph.params
        p = GraphParams(gp.D, gp.g_graph, gp.g_cell, gp.threshold, gp.delay_ortho, gp.delay_anti,
                        gp.amplitude, gp.duration, gp.radius, int(gp.two_way), 0, 0.0)
        rc = lib().orc_sim_attach_graph(self._h, keep[0].shape[0], _ptr(keep[0]), keep[1].shape[0], _ptr(keep[1]),
                                        None if keep[2] is None else _ptr(keep[2]), _ptr(keep[3]), _ptr(keep[4]),
                                        keep[5].size, _ptr(keep[5]), _ptr(keep[6]), _ptr(keep[7]), ctypes.byref(p))
        if rc:
            raise ValueError(f"oracle graph rejected (code {rc})")
        self.n_graph = keep[0].shape[0]

    @property
    def graph_substeps(self) -> int:
        return int(lib().orc_sim_graph_substeps(self._h))

    def graph_get(self, var: int) -> np.ndarray:
        out = np.zeros(self.n_graph)
        lib().orc_sim_graph_get_var(self._h, int(var), _ptr(out))
        return out

    def graph_set(self, var: int, values) -> None:
        v = np.ascontiguousarray(values, dtype=np.float64)
        lib().orc_sim_graph_set_var(self._h, int(var), _ptr(v))

    def graph_laplacian(self, W) -> np.ndarray:
        W = np.ascontiguousarray(W, dtype=np.float64)
        out = np.zeros(self.n_graph)
        lib().orc_sim_graph_laplacian(self._h, _ptr(W), _ptr(out))
        return out

    def graph_activation_times(self) -> np.ndarray:
        out = np.zeros(self.n_graph)
        lib().orc_sim_graph_get_act(self._h, _ptr(out))
        return out
