"""Python binding of ``libep.so`` (include/ep.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
converts numpy arrays and Python values to the C structures, routes device
allocations to PyTorch's caching allocator and passes PyTorch's current CUDA
stream. If the library is missing it raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libep.so")

EP_OK, EP_EINVAL, EP_ENOMEM, EP_EMESH, EP_EUNSTABLE, EP_ENONFINITE, EP_ETIMEOUT, EP_ECUDA, EP_ESTATE = range(9)
EP_TP06, EP_CRN, EP_STEWART = 0, 1, 2
EP_FP32_MIXED, EP_FP64_PLAIN = 0, 1
EP_INTEGRATOR_FE, EP_INTEGRATOR_AB2 = 0, 1
MAX_SETS, MAX_STIM = 16, 8
_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "EMESH", 4: "EUNSTABLE", 5: "ENONFINITE", 6: "ETIMEOUT",
           7: "ECUDA", 8: "ESTATE"}


class EPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ep error {code} ({_STATUS.get(code, '?')}): {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("n_cells", ctypes.c_int64),
                ("tet", ctypes.c_void_p), ("cell_model", ctypes.c_void_p), ("param_set", ctypes.c_void_p),
                ("stim_mask", ctypes.c_void_p), ("fibre", ctypes.c_void_p), ("n_tris", ctypes.c_int64),
                ("tri", ctypes.c_void_p), ("index_width", ctypes.c_int32), ("pad", ctypes.c_int32)]


class CellParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("reserved", ctypes.c_int32), ("D_l", ctypes.c_double),
                ("D_t", ctypes.c_double), ("gks_scale", ctypes.c_double), ("gkr_scale", ctypes.c_double),
                ("K_o", ctypes.c_double)]


class Stimulus(ctypes.Structure):
    _fields_ = [("amplitude", ctypes.c_double), ("t_on", ctypes.c_double), ("duration", ctypes.c_double),
                ("period", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("precision", ctypes.c_int32), ("n_sets", ctypes.c_int32),
                ("sets", CellParams * MAX_SETS), ("n_stim", ctypes.c_int32), ("integrator", ctypes.c_int32),
                ("stim", Stimulus * MAX_STIM), ("threshold", ctypes.c_double)]


class BidoSolver(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("atol", ctypes.c_double), ("restart", ctypes.c_int32),
                ("reorth", ctypes.c_int32), ("max_iter", ctypes.c_int64), ("barrier_limit_s", ctypes.c_double)]


class BidoStats(ctypes.Structure):
    _fields_ = [("last_iters", ctypes.c_int64), ("total_iters", ctypes.c_int64), ("solves", ctypes.c_int64),
                ("last_res", ctypes.c_double), ("last_bnorm", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 5), ("failed", ctypes.c_int32), ("timeout", ctypes.c_int32)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("n_edges", ctypes.c_int64),
                ("edges", ctypes.c_void_p), ("edge_D", ctypes.c_void_p), ("node_model", ctypes.c_void_p),
                ("node_param_set", ctypes.c_void_p), ("node_stim_mask", ctypes.c_void_p),
                ("n_junctions", ctypes.c_int64), ("junction_node", ctypes.c_void_p),
                ("junction_cell", ctypes.c_void_p), ("junction_mode", ctypes.c_void_p)]


class GraphParamsC(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("g_graph", ctypes.c_double), ("g_cell", ctypes.c_double),
                ("threshold", ctypes.c_double), ("delay_ortho", ctypes.c_double), ("delay_anti", ctypes.c_double),
                ("amplitude", ctypes.c_double), ("duration", ctypes.c_double), ("radius", ctypes.c_double),
                ("two_way", ctypes.c_int32), ("default_mode", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

# every symbol declared in include/ep.h
EP_GRAPH_SUBSTEPS_LAUNCHES, EP_GRAPH_SUBSTEPS_LOCAL = 0, 1
NOALLOC_MAX_NODES = 2097152
NOALLOC_MAX_CELLS = 16777216

EXPORTS = ["ep_context_create", "ep_context_set_stream", "ep_context_destroy", "ep_last_error",
           "ep_mesh_create", "ep_params_set", "ep_step", "ep_read_state", "ep_write_state",
           "ep_activation_times", "ep_reset_activation", "ep_step_index", "ep_set_step_index",
           "ep_check_finite", "ep_job_info", "ep_estimate_bytes", "ep_job_destroy", "ep_model_nvar",
           "ep_model_varname", "ep_plan_inspect", "ep_time_kernels",
           "ep_step_noalloc", "ep_autotune", "ep_set_cell_variant", "ep_plan_create", "ep_plan_bytes",
           "ep_plan_info", "ep_plan_destroy", "ep_job_create", "ep_graph_attach", "ep_graph_read_state",
           "ep_graph_write_state", "ep_graph_activation_times", "ep_graph_info", "ep_alu_peaks",
           "ep_bidomain_enable", "ep_bidomain_disable", "ep_bidomain_read_ve", "ep_bidomain_write_ve",
           "ep_bidomain_stats", "ep_clear_error", "ep_set_graph_kernel", "ep_read_state_f32",
           "ep_write_state_f32", "ep_activation_times_f32", "ep_model_var_compensated"]

_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def load():
    """Load libep.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2112_12854_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "ep_context_create": ([ALLOC_FN, FREE_FN, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
        "ep_context_set_stream": ([_P, _P], ctypes.c_int),
        "ep_context_destroy": ([_P], ctypes.c_int),
        "ep_last_error": ([_P], ctypes.c_char_p),
        "ep_mesh_create": ([_P, ctypes.POINTER(MeshDesc), ctypes.POINTER(_P)], ctypes.c_int),
        "ep_params_set": ([_P, ctypes.POINTER(Params)], ctypes.c_int),
        "ep_step": ([ctypes.POINTER(_P), ctypes.c_int32, _I64], ctypes.c_int),
        "ep_read_state": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _I64], ctypes.c_int),
        "ep_write_state": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _I64], ctypes.c_int),
        "ep_activation_times": ([_P, _P, _I64], ctypes.c_int),
        "ep_read_state_f32": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _I64], ctypes.c_int),
        "ep_write_state_f32": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _I64], ctypes.c_int),
        "ep_activation_times_f32": ([_P, _P, _I64], ctypes.c_int),
        "ep_model_var_compensated": ([ctypes.c_int32, ctypes.c_int32], ctypes.c_int32),
        "ep_reset_activation": ([_P], ctypes.c_int),
        "ep_step_index": ([_P, ctypes.POINTER(_I64)], ctypes.c_int),
        "ep_set_step_index": ([_P, _I64], ctypes.c_int),
        "ep_check_finite": ([_P], ctypes.c_int),
        "ep_clear_error": ([_P], ctypes.c_int),
        "ep_set_graph_kernel": ([_P, ctypes.c_int32], ctypes.c_int),
        "ep_job_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                         ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
                        ctypes.c_int),
        "ep_estimate_bytes": ([_I64, _I64, ctypes.c_int32], _I64),
        "ep_job_destroy": ([_P], ctypes.c_int),
        "ep_model_nvar": ([ctypes.c_int32], ctypes.c_int32),
        "ep_model_varname": ([ctypes.c_int32, ctypes.c_int32], ctypes.c_char_p),
        "ep_step_noalloc": ([_P, _I64], ctypes.c_int),
        "ep_graph_attach": ([_P, ctypes.POINTER(GraphDesc), ctypes.POINTER(GraphParamsC)], ctypes.c_int),
        "ep_graph_read_state": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _I64], ctypes.c_int),
        "ep_graph_write_state": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _I64], ctypes.c_int),
        "ep_graph_activation_times": ([_P, _P, _I64], ctypes.c_int),
        "ep_graph_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_I64)],
                          ctypes.c_int),
        "ep_plan_create": ([ctypes.POINTER(MeshDesc), ctypes.POINTER(Params), ctypes.POINTER(_P)], ctypes.c_int),
        "ep_plan_bytes": ([_P], _I64),
        "ep_plan_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "ep_plan_destroy": ([_P], ctypes.c_int),
        "ep_job_create": ([_P, _P, ctypes.POINTER(_P)], ctypes.c_int),
        "ep_autotune": ([ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32, _P, _P], ctypes.c_int),
        "ep_set_cell_variant": ([_P, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "ep_alu_peaks": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "ep_bidomain_enable": ([_P, _P, _P, ctypes.c_int32, ctypes.POINTER(BidoSolver)], ctypes.c_int),
        "ep_bidomain_disable": ([_P], ctypes.c_int),
        "ep_bidomain_read_ve": ([_P, _P, _I64], ctypes.c_int),
        "ep_bidomain_write_ve": ([_P, _P, _I64], ctypes.c_int),
        "ep_bidomain_stats": ([_P, ctypes.POINTER(BidoStats)], ctypes.c_int),
        "ep_time_kernels": ([ctypes.POINTER(_P), ctypes.c_int32, _I64, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "ep_plan_inspect": ([ctypes.POINTER(MeshDesc), ctypes.POINTER(Params)] + [_P] * 10
                            + [ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def model_varnames(model: int) -> list[str]:
    L = load()
    return [L.ep_model_varname(model, k).decode() for k in range(L.ep_model_nvar(model))]


def model_var_compensated(model: int) -> list:
    """Per variable of the model: True where an FP32 job stores it as a
    compensated sum (transferred in FP64 only)."""
    L = load()
    return [bool(L.ep_model_var_compensated(model, k)) for k in range(L.ep_model_nvar(model))]


def estimate_bytes(n_cells: int, n_nodes: int, precision: int = EP_FP32_MIXED) -> int:
    return int(load().ep_estimate_bytes(n_cells, n_nodes, precision))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class Context:
    """A library context on the current CUDA device. Device memory comes from
    PyTorch's caching allocator (or cudaMalloc with ``torch_allocator=False``);
    work is enqueued on ``stream`` (default: PyTorch's current stream)."""

    def __init__(self, stream=None, torch_allocator: bool = True):
        import torch
        L = load()
        self._torch = torch
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._stream_ptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        if torch_allocator:
            dev, st = self.device, stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:  # out of memory: the library reports EP_ENOMEM
                    return None

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc, self._free = ALLOC_FN(_alloc), FREE_FN(_free)
        else:
            self._alloc, self._free = ctypes.cast(None, ALLOC_FN), ctypes.cast(None, FREE_FN)
        h = _P()
        rc = L.ep_context_create(self._alloc, self._free, None, self._stream_ptr, ctypes.byref(h))
        if rc:
            raise EPError(rc, L.ep_last_error(None).decode())
        self._h = h
        self.jobs = set()

    def check(self, rc):
        if rc:
            raise EPError(rc, load().ep_last_error(self._h).decode())

    def set_graph_kernel(self, mode: int):
        """EP_GRAPH_SUBSTEPS_LOCAL (one launch for all substeps, the default) or
        EP_GRAPH_SUBSTEPS_LAUNCHES (one launch per substep)."""
        self.check(load().ep_set_graph_kernel(self._h, int(mode)))

    def clear_error(self):
        """Forget a step kernel's bounded wait that gave up (ep_clear_error)."""
        self.check(load().ep_clear_error(self._h))

    def close(self):
        for j in list(self.jobs):
            j.destroy()
        if getattr(self, "_h", None):
            self.check(load().ep_context_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mesh(self, xyz, tets, *, cell_model=None, param_set=None, stim_mask=None, fibre=None, tris=None,
             index_width=0) -> "Job":
        return Job(self, xyz, tets, cell_model=cell_model, param_set=param_set, stim_mask=stim_mask,
                   fibre=fibre, tris=tris, index_width=index_width)


def make_params(dt, sets, stimuli=(), *, precision=EP_FP32_MIXED, threshold=-20.0,
                integrator=0) -> Params:
    """sets: objects with variant, D_l, D_t, gks_scale, gkr_scale, K_o;
    stimuli: objects with amplitude, t_on, duration, period; integrator
    EP_INTEGRATOR_FE (0) or EP_INTEGRATOR_AB2 (1) for the non-gating variables."""
    p = Params()
    p.dt = float(dt)
    p.precision = int(precision)
    p.integrator = int(integrator)
    p.n_sets = len(sets)
    if not 1 <= len(sets) <= MAX_SETS or len(stimuli) > MAX_STIM:
        raise ValueError("1..16 parameter sets and at most 8 stimuli")
    for k, s in enumerate(sets):
        p.sets[k] = CellParams(int(getattr(s, "variant", 0)), 0, float(s.D_l), float(s.D_t),
                               float(getattr(s, "gks_scale", 1.0)), float(getattr(s, "gkr_scale", 1.0)),
                               float(getattr(s, "K_o", 5.4)))
    p.n_stim = len(stimuli)
    for k, s in enumerate(stimuli):
        p.stim[k] = Stimulus(float(s.amplitude), float(s.t_on), float(s.duration), float(getattr(s, "period", 0.0)))
    p.threshold = float(threshold)
    return p


def _mesh_desc(xyz, tets, cell_model=None, param_set=None, stim_mask=None, fibre=None, tris=None, index_width=0):
    """ep_mesh_desc of numpy inputs (tets, then the shell triangles `tris`);
    returns (desc, arrays to keep alive)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(np.reshape(tets, (-1, 4)), dtype=np.int32)
    tris = np.ascontiguousarray(np.zeros((0, 3)) if tris is None else np.reshape(tris, (-1, 3)), dtype=np.int32)
    n = tets.shape[0] + tris.shape[0]
    keep = [xyz, tets, tris]
    d = MeshDesc()
    d.n_nodes, d.xyz, d.n_cells, d.tet = xyz.shape[0], _ptr(xyz), tets.shape[0], _ptr(tets)
    d.n_tris, d.tri = tris.shape[0], _ptr(tris)
    d.index_width = int(index_width)
    for name, arr, dt, width in (("cell_model", cell_model, np.uint8, 1), ("param_set", param_set, np.uint8, 1),
                                 ("stim_mask", stim_mask, np.uint8, 1), ("fibre", fibre, np.float64, 3)):
        if arr is None:
            setattr(d, name, None)
            continue
        a = np.ascontiguousarray(arr, dtype=dt)
        if a.size != n * width:
            raise ValueError(f"{name} must have {n * width} entries")
        keep.append(a)
        setattr(d, name, _ptr(a))
    return d, keep


class Plan:
    """Host-only job preparation (ep_plan_create): no device, no context,
    safe to build in worker threads while the GPU steps other jobs."""

    def __init__(self, xyz, tets, params: Params | None = None, *, cell_model=None, param_set=None,
                 stim_mask=None, fibre=None, tris=None, index_width=0):
        L = load()
        d, keep = _mesh_desc(xyz, tets, cell_model, param_set, stim_mask, fibre, tris, index_width)
        h = _P()
        rc = L.ep_plan_create(ctypes.byref(d), ctypes.byref(params) if params is not None else None,
                              ctypes.byref(h))
        if rc:
            raise EPError(rc, L.ep_last_error(None).decode())
        self._h = h
        self.params = params
        a, b, iw, niw = _I64(), _I64(), ctypes.c_int32(), ctypes.c_int32()
        L.ep_plan_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(iw), ctypes.byref(niw))
        self.n_cells, self.n_nodes = int(a.value), int(b.value)
        self.index_width, self.node_index_width = int(iw.value), int(niw.value)
        self.device_bytes = int(L.ep_plan_bytes(h))

    def destroy(self):
        if getattr(self, "_h", None):
            load().ep_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        self.destroy()


class Job:
    def __init__(self, ctx: Context, xyz=None, tets=None, *, plan: Plan | None = None, cell_model=None,
                 param_set=None, stim_mask=None, fibre=None, tris=None, index_width=0):
        L = load()
        self.ctx = ctx
        h = _P()
        if plan is not None:
            ctx.check(L.ep_job_create(ctx._h, plan._h, ctypes.byref(h)))
            self.n_cells = plan.n_cells
            if plan.params is not None:
                self.params = plan.params
        else:
            d, keep = _mesh_desc(xyz, tets, cell_model, param_set, stim_mask, fibre, tris, index_width)
            ctx.check(L.ep_mesh_create(ctx._h, ctypes.byref(d), ctypes.byref(h)))
            self.n_cells = int(d.n_cells) + int(d.n_tris)
        self._h = h
        ctx.jobs.add(self)

    def set_params(self, params: Params):
        self.ctx.check(load().ep_params_set(self._h, ctypes.byref(params)))
        self.params = params

    def step(self, n_steps: int):
        step([self], n_steps)

    def read(self, var, model: int = EP_TP06, out=None) -> np.ndarray:
        if isinstance(var, str):
            var = model_varnames(model).index(var)
        if out is None:
            out = np.empty(self.n_cells, np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.n_cells
        self.ctx.check(load().ep_read_state(self._h, model, var, _ptr(out), self.n_cells))
        return out

    def write(self, var, values, model: int = EP_TP06):
        if isinstance(var, str):
            var = model_varnames(model).index(var)
        v = np.ascontiguousarray(values, dtype=np.float64)
        self.ctx.check(load().ep_write_state(self._h, model, var, _ptr(v), self.n_cells))

    def read_f32(self, var, model: int = EP_TP06, out=None) -> np.ndarray:
        """ep_read_state_f32: a variable an FP32 job stores in FP32, exactly."""
        if isinstance(var, str):
            var = model_varnames(model).index(var)
        if out is None:
            out = np.empty(self.n_cells, np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == self.n_cells
        self.ctx.check(load().ep_read_state_f32(self._h, model, var, _ptr(out), self.n_cells))
        return out

    def write_f32(self, var, values, model: int = EP_TP06):
        """ep_write_state_f32."""
        if isinstance(var, str):
            var = model_varnames(model).index(var)
        v = np.ascontiguousarray(values, dtype=np.float32)
        self.ctx.check(load().ep_write_state_f32(self._h, model, var, _ptr(v), self.n_cells))

    @property
    def V(self) -> np.ndarray:
        return self.read(0)

    def activation_times(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n_cells, np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.n_cells
        self.ctx.check(load().ep_activation_times(self._h, _ptr(out), self.n_cells))
        return out

    def activation_times_f32(self, out=None) -> np.ndarray:
        """ep_activation_times_f32 (an FP32 job)."""
        if out is None:
            out = np.empty(self.n_cells, np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == self.n_cells
        self.ctx.check(load().ep_activation_times_f32(self._h, _ptr(out), self.n_cells))
        return out

    def reset_activation(self):
        self.ctx.check(load().ep_reset_activation(self._h))

    @property
    def step_index(self) -> int:
        v = _I64()
        self.ctx.check(load().ep_step_index(self._h, ctypes.byref(v)))
        return int(v.value)

    @step_index.setter
    def step_index(self, n):
        self.ctx.check(load().ep_set_step_index(self._h, int(n)))

    def check_finite(self) -> bool:
        rc = load().ep_check_finite(self._h)
        if rc == EP_ENONFINITE:
            return False
        self.ctx.check(rc)
        return True

    def info(self) -> dict:
        a, b, c, d, iw, niw = _I64(), _I64(), _I64(), _I64(), ctypes.c_int32(), ctypes.c_int32()
        self.ctx.check(load().ep_job_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(d), ctypes.byref(iw), ctypes.byref(niw)))
        return dict(n_cells=a.value, n_nodes=b.value, n_interior_faces=c.value, device_bytes=d.value,
                    index_width=iw.value, node_index_width=niw.value)

    def attach_graph(self, graph, *, node_model=None):
        """Attach a conduction graph (an object like ``workloads.Graph``:
        xyz, edges, edge_D, param_set, stim_mask, junction_node/cell/mode,
        params). node_model defaults to the models of the graph's parameter
        sets when ``model_of_set`` is given on the graph, else Stewart."""
        L = load()
        keep = []

        def arr(a, dt):
            if a is None:
                return None
            b = np.ascontiguousarray(a, dtype=dt)
            keep.append(b)
            return _ptr(b)
        d = GraphDesc()
        d.n_nodes = int(np.asarray(graph.xyz).shape[0])
        d.xyz = arr(graph.xyz, np.float64)
        d.n_edges = int(np.asarray(graph.edges).reshape(-1, 2).shape[0])
        d.edges = arr(np.asarray(graph.edges).reshape(-1, 2), np.int32)
        d.edge_D = arr(graph.edge_D, np.float64)
        d.node_model = arr(node_model, np.uint8)
        d.node_param_set = arr(graph.param_set, np.uint8)
        d.node_stim_mask = arr(graph.stim_mask, np.uint8)
        d.n_junctions = int(np.asarray(graph.junction_node).size)
        d.junction_node = arr(graph.junction_node, np.int32)
        d.junction_cell = arr(graph.junction_cell, np.int32)
        d.junction_mode = arr(graph.junction_mode, np.uint8)
        gp = graph.params
        p = GraphParamsC(gp.D, gp.g_graph, gp.g_cell, gp.threshold, gp.delay_ortho, gp.delay_anti, gp.amplitude,
                         gp.duration, gp.radius, int(gp.two_way), 0)
        self.ctx.check(L.ep_graph_attach(self._h, ctypes.byref(d), ctypes.byref(p)))
        self.n_graph = d.n_nodes

    def graph_read(self, var, model: int = EP_STEWART, out=None) -> np.ndarray:
        if isinstance(var, str):
            var = model_varnames(model).index(var)
        out = np.empty(self.n_graph, np.float64) if out is None else out
        self.ctx.check(load().ep_graph_read_state(self._h, model, var, _ptr(out), self.n_graph))
        return out

    def graph_write(self, var, values, model: int = EP_STEWART):
        v = np.ascontiguousarray(values, dtype=np.float64)
        self.ctx.check(load().ep_graph_write_state(self._h, model, int(var), _ptr(v), self.n_graph))

    def graph_activation_times(self) -> np.ndarray:
        out = np.empty(self.n_graph, np.float64)
        self.ctx.check(load().ep_graph_activation_times(self._h, _ptr(out), self.n_graph))
        return out

    def graph_info(self) -> dict:
        a, b, c = _I64(), ctypes.c_int32(), _I64()
        self.ctx.check(load().ep_graph_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(n_nodes=a.value, substeps=b.value, n_junctions=c.value)

    def enable_bidomain(self, De_l, De_t, *, tol=None, atol=None, restart=12, reorth=0, max_iter=2000,
                        n_sets=None, barrier_limit_s=0.0):
        """Bidomain model (ep_bidomain_enable): De_l, De_t are the
        extracellular diffusivities, scalars or one per parameter set; the
        parameter sets' own (D_l, D_t) become the intracellular ones. tol /
        atol None take the library's defaults for the job's precision."""
        params = getattr(self, "params", None)
        if n_sets is None:
            n_sets = params.n_sets if params is not None else np.size(De_l)
        el = np.ascontiguousarray(np.broadcast_to(np.asarray(De_l, np.float64), (n_sets,)))
        et = np.ascontiguousarray(np.broadcast_to(np.asarray(De_t, np.float64), (n_sets,)))
        sv = None
        if (tol is not None or atol is not None or restart != 12 or reorth != 0 or max_iter != 2000
                or barrier_limit_s > 0.0):
            plain = params is not None and params.precision == EP_FP64_PLAIN
            sv = BidoSolver(float(tol if tol is not None else (1e-11 if plain else 1e-5)),
                            float(atol if atol is not None else (1e-11 if plain else 1e-3)),
                            int(restart), int(reorth), int(max_iter), float(barrier_limit_s))
        self.ctx.check(load().ep_bidomain_enable(self._h, _ptr(el), _ptr(et), int(n_sets),
                                                 ctypes.byref(sv) if sv is not None else None))

    def disable_bidomain(self):
        self.ctx.check(load().ep_bidomain_disable(self._h))

    @property
    def ve(self) -> np.ndarray:
        out = np.empty(self.n_cells, np.float64)
        self.ctx.check(load().ep_bidomain_read_ve(self._h, _ptr(out), self.n_cells))
        return out

    @ve.setter
    def ve(self, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.size == self.n_cells
        self.ctx.check(load().ep_bidomain_write_ve(self._h, _ptr(v), self.n_cells))

    def bidomain_stats(self) -> dict:
        st = BidoStats()
        self.ctx.check(load().ep_bidomain_stats(self._h, ctypes.byref(st)))
        return {"last_iters": st.last_iters, "total_iters": st.total_iters, "solves": st.solves,
                "last_res": st.last_res, "last_bnorm": st.last_bnorm, "alg_bytes": st.alg_bytes,
                "phase_ms": list(st.phase_ms), "failed": bool(st.failed), "timeout": bool(st.timeout)}

    def destroy(self):
        if getattr(self, "_h", None):
            self.ctx.check(load().ep_job_destroy(self._h))
            self._h = None
            self.ctx.jobs.discard(self)


def step(jobs, n_steps: int):
    """Advance all jobs by n_steps in shared batched launches (ep_step)."""
    arr = (_P * len(jobs))(*[j._h for j in jobs])
    jobs[0].ctx.check(load().ep_step(arr, len(jobs), int(n_steps)))


def step_noalloc(job, n_steps: int):
    """Advance one job by n_steps through ep_step_noalloc (no device allocation;
    node values in the library's static device array, see include/ep.h)."""
    job.ctx.check(load().ep_step_noalloc(job._h, int(n_steps)))


N_CELL_VARIANTS = 12


def autotune(jobs, steps_per_variant: int = 10):
    """Pick the fastest cell-kernel launch shape per precision (ep_autotune).
    Advances the jobs by N_CELL_VARIANTS * steps_per_variant real steps.
    Returns (chosen[2], ms[2][N_CELL_VARIANTS])."""
    arr = (_P * len(jobs))(*[j._h for j in jobs])
    chosen = np.zeros(2, np.int32)
    ms = np.zeros(2 * N_CELL_VARIANTS, np.float64)
    jobs[0].ctx.check(load().ep_autotune(arr, len(jobs), int(steps_per_variant), _ptr(chosen), _ptr(ms)))
    return chosen, ms.reshape(2, N_CELL_VARIANTS)


def set_cell_variant(ctx: "Context", precision: int, variant: int):
    ctx.check(load().ep_set_cell_variant(ctx._h, int(precision), int(variant)))


def time_kernels(jobs, n_steps: int):
    """Advance the jobs by n_steps with CUDA events around each launch;
    returns the mean (node_ms, cell_ms) device time per step."""
    arr = (_P * len(jobs))(*[j._h for j in jobs])
    a, b = ctypes.c_double(), ctypes.c_double()
    jobs[0].ctx.check(load().ep_time_kernels(arr, len(jobs), int(n_steps), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def alu_peaks(ctx) -> dict:
    """Measured issue rates of the FP32 FMA, MUFU ex2 and FP64 FMA pipes
    (operations per second; an FMA counts two flops)."""
    out = (ctypes.c_double * 3)()
    ctx.check(load().ep_alu_peaks(ctx._h, out))
    return {"fp32_fma_flops": out[0], "mufu_ex2_ops": out[1], "fp64_fma_flops": out[2]}


def case_cell_model(case):
    return np.array([case.param_sets[k].model for k in range(len(case.param_sets))], np.uint8)[case.param_set]


def plan_from_case(case, *, precision=EP_FP32_MIXED, integrator=0, index_width=0) -> Plan:
    """Host-only plan of a ``workloads.TissueCase`` (mesh + parameters)."""
    params = make_params(case.dt, case.param_sets, case.stimuli, precision=precision, threshold=case.threshold,
                         integrator=integrator)
    return Plan(case.xyz, case.tets, params, cell_model=case_cell_model(case), param_set=case.param_set,
                stim_mask=case.stim_mask, fibre=case.fibre, tris=getattr(case, "tris", None),
                index_width=index_width)


def job_from_case(ctx: Context, case, *, precision=EP_FP32_MIXED, cell_model=None, integrator=0,
                  index_width=0) -> Job:
    """Create a job from a ``workloads.TissueCase`` and set its parameters."""
    if cell_model is None:
        cell_model = case_cell_model(case)
    j = ctx.mesh(case.xyz, case.tets, cell_model=cell_model, param_set=case.param_set,
                 stim_mask=case.stim_mask, fibre=case.fibre, tris=getattr(case, "tris", None),
                 index_width=index_width)
    j.set_params(make_params(case.dt, case.param_sets, case.stimuli, precision=precision,
                             threshold=case.threshold, integrator=integrator))
    return j


def plan_inspect(xyz, tets, params: Params, *, cell_model=None, param_set=None, fibre=None, tris=None) -> dict:
    """Run the host planner only (no GPU) and return its folded operator
    (cells: the tets, then the shell triangles)."""
    L = load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(np.reshape(tets, (-1, 4)), dtype=np.int32)
    tris = np.ascontiguousarray(np.zeros((0, 3)) if tris is None else np.reshape(tris, (-1, 3)), dtype=np.int32)
    n, nn = tets.shape[0] + tris.shape[0], xyz.shape[0]
    keep = [tris]
    d = MeshDesc()
    d.n_nodes, d.xyz, d.n_cells, d.tet = nn, _ptr(xyz), tets.shape[0], _ptr(tets)
    d.n_tris, d.tri = tris.shape[0], _ptr(tris)
    for name, arr, dt in (("cell_model", cell_model, np.uint8), ("param_set", param_set, np.uint8),
                          ("fibre", fibre, np.float64)):
        if arr is None:
            setattr(d, name, None)
        else:
            a = np.ascontiguousarray(arr, dtype=dt)
            keep.append(a)
            setattr(d, name, _ptr(a))
    d.stim_mask = None
    out = dict(cell_order=np.zeros(n, np.int64), tet=np.zeros(4 * n, np.int32), opp=np.zeros(4 * n, np.int32),
               nbr=np.zeros(4 * n, np.int32), wa=np.zeros(4 * n), wb=np.zeros(4 * n), q=np.zeros(4 * n),
               n2c_ptr=np.zeros(nn + 1, np.int64), n2c=np.zeros(4 * n, np.int32), nw=np.zeros(4 * n))
    rho = ctypes.c_double(0.0)
    rc = L.ep_plan_inspect(ctypes.byref(d), ctypes.byref(params), *[_ptr(out[k]) for k in
                           ("cell_order", "tet", "opp", "nbr", "wa", "wb", "q", "n2c_ptr", "n2c", "nw")],
                           ctypes.byref(rho))
    if rc:
        raise EPError(rc, L.ep_last_error(None).decode())
    out["rho_bound"] = rho.value
    return out
