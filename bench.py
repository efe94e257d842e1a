"""Benchmark of the monodomain finite-volume step on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (``ours``): the ventricular wedge slab, 50 x 50 x 10 mm at 0.25 mm
(200 x 200 x 40 cubes x 6 tets = 9.6M cells), fibre angle rotating from -60
deg (endocardium) to +60 deg (epicardium), TP06 endo / M / epi variants in
depth thirds, corner stimulus, dt = 0.02 ms; seeded synthetic input shaped
like the paper's slab benchmark (Sec. 4). A "step" is one time step of every
cell: the node-value launch and the fused cell launch. ``value`` is
cell-updates/s of the FP32 path (FP64 accumulation of [Na]i, [K]i, [Ca]SR)
with the state resident in HBM; the plain FP64 path is timed beside it on the
same workload. Under torchrun each rank runs its own replica (the path has no
exchange step); ``value`` sums the ranks' cell-updates over the slowest
rank's time.

``--impl reference`` times the FP64 CPU oracle as it stands on this host's
cores, on a bounded crop of the same workload (same construction, fewer
cubes), one oracle time step per bench step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

METRIC = "cell-updates/s FP32 batched vs FP64 plain (same GPU, ≤1 mV); p50/p99 job latency"
UNIT = "cell-updates/s"
WEDGE = dict(nx=200, ny=200, nz=40, h=0.25)
CROP = dict(nx=50, ny=50, nz=10, h=0.25)       # oracle sample: same construction, 150k cells
OUTPUT_EVERY = 250                              # V read back every 5 ms of simulated time (e2e)
# Algorithmic bytes per cell-update of the fused cell kernel (TP06, FP32 mixed):
#   gather indices: 8 node + 4 neighbour indices, as 16-bit offsets (24 B) or 32-bit (48 B)
#   folded coefficients wa, wb, q (3 x float4) = 48
#   own V read 4, pset + stim mask 2, state read 15 x 4 + 3 x 8 = 84
#   V^{n+1} write 4, state write 84
# (node-value and neighbour-potential gathers are L2 hits by design and not counted)
def cell_bytes(index_width):
    return (24 if index_width == 16 else 48) + 48 + 4 + 2 + 84 + 4 + 84


# node kernel: sliced-ELL entries (a 2- or 4-byte cell index + 4-byte weight) per incidence
# (4 per cell), plus the node-value write (N_nodes / N_cells x 4 bytes)
def node_bytes_per_incidence(index_width):
    return (2 if index_width == 16 else 4) + 4


# A second byte floor, of the shared-face form of the step (TP06, mixed precision: state,
# cell->node indices, node CSR, face coefficients read once per face, volume and parameter
# byte): 277 B per cell-update, of which the node CSR is 32 B; the cell kernel's part is the
# other 245 B.
FACE_STEP_FLOOR = 277
FACE_CELL_FLOOR = 277 - 32


# launch-shape variants that do the whole step in one launch (ep_autotune)
FUSED_VARIANTS = (8, 9)


def wedge_case(dims):
    return w.wedge_case(nx=dims["nx"], ny=dims["ny"], nz=dims["nz"], h=dims["h"], n_steps=20000)


# Sources the node and cell kernels are compiled from (the profiles under
# profiles/ record the hash of these files at capture time).
STEP_KERNEL_SOURCES = ("kernels.cu", "kernels_tab.cu", "kernels_f64.cu", "cellstep.cuh", "kernels.h", "devtypes.h",
                       "cellmath.cuh", "ttcells.cuh", "crncell.cuh", "varmap.h", "nodesum.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2112_12854_b300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profile_value(fname, key):
    """A per-cell figure recorded in a committed ncu summary under profiles/,
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    m_v = re.search(key + r":\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_v or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_v.group(1))


def traffic_from_profile(n_cells):
    """DRAM bytes of one cell-kernel launch (FP32) from the ncu summary."""
    b = profile_value("cell_kernel_wedge.md", "dram_bytes_per_cell")
    return None if b is None else b * n_cells


def alu_side(n_cells, cell_ms, alu):
    """The FP32 cell kernel against its two ALU roofs: FP32 FMA-pipe and
    MUFU (XU-pipe) thread operations per cell, counted by ncu on the crop
    (committed summary, current kernel source only), times the cell-update
    rate, over the measured issue rates of those pipes (ep_alu_peaks)."""
    fma = profile_value("cell_kernel_wedge.md", "fma_pipe_thread_ops_per_cell")
    xu = profile_value("cell_kernel_wedge.md", "xu_pipe_thread_ops_per_cell")
    rate = n_cells / (cell_ms * 1e-3)
    out = {"source": "ncu instruction counts per pipe on the crop (profiles/cell_kernel_wedge.md) x "
                     "cell-updates/s; peaks from ep_alu_peaks"}
    if fma is not None:
        # an FMA-pipe instruction counts one operation; the measured FMA peak counts two flops per FMA
        ach = fma * rate / 1e12
        pk = alu["fp32_fma_flops"] / 2e12
        out["fma"] = {"achieved_tops": ach, "peak_tops": pk, "frac": ach / pk, "ops_per_cell": fma}
    if xu is not None:
        ach = xu * rate / 1e12
        pk = alu["mufu_ex2_ops"] / 1e12
        out["mufu"] = {"achieved_tops": ach, "peak_tops": pk, "frac": ach / pk, "ops_per_cell": xu}
    return out


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, smax, reasons = [], [], set()
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def oracle_throughput(dims, budget_s, max_steps=None):
    """Time the FP64 oracle on a crop of the workload; returns (cell-updates/s, steps, cells, cores)."""
    import oracle
    case = wedge_case(dims)
    s = oracle.Sim(case)
    s.run(1)
    t0 = time.perf_counter()
    steps = 0
    while True:
        s.run(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    cores = oracle.set_threads(0)     # the OpenMP thread count the oracle ran with
    return case.n_cells * steps / el, steps, case.n_cells, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    case = wedge_case(CROP)
    s = oracle.Sim(case)
    # A fresh simulation takes about a second of steps to reach its steady speed on the host
    # cores (measured on the GPU machine: 8.1-8.5 ms per step over the 20 steps after 5 warm-up
    # steps, 5.9 ms over 200, also after a second of steps on another simulation): run it
    # for 1 s untimed first, so that the timed steps measure the oracle, not the ramp.
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        s.run(1)
    for _ in range(args.warmup):
        s.run(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.run(1)
    el = time.perf_counter() - t0
    cores = oracle.set_threads(0)
    val = case.n_cells * args.steps / el
    sample = (f"oracle (FP64 C, OpenMP) on a crop of the wedge workload: {CROP['nx']}x{CROP['ny']}x{CROP['nz']} "
              f"cubes x 6 = {case.n_cells} cells, one time step per bench step, after 1 s of untimed "
              f"steps and the warm-up steps")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "ventricular wedge slab crop (oracle sample)",
                                            "cells": case.n_cells, "dt_ms": case.dt},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_beat(ctx, args, dims, stream, torch):
    """The headline workload over one whole beat: a fresh FP32 job from the
    resting state, stimulated at t = 0, stepped through args.beat_steps steps
    (400 ms at dt = 0.02 ms) in chunks of 1000 steps timed with CUDA events;
    reports the whole-beat rate and the steady window of the 1000 steps in
    the middle of the beat. The launch shape is the context's (autotuned)."""
    from paper_2112_12854_b300 import ep
    case = wedge_case(dims)
    job = ep.job_from_case(ctx, case, precision=ep.EP_FP32_MIXED)
    torch.cuda.synchronize()
    chunk = 1000                    # the first chunk includes the capture of the step graph (~1 ms)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.beat_steps // chunk + 1)]
    evs[0].record(stream)
    for k in range(args.beat_steps // chunk):
        job.step(chunk)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(len(evs) - 1)]
    total = sum(ms)
    mid = ms[len(ms) // 2]
    act = job.activation_times()
    finite = job.check_finite()
    job.destroy()
    n = case.n_cells
    steps = chunk * len(ms)
    return {"steps": steps, "simulated_ms": steps * case.dt, "ms_per_step": total / steps,
            "cell_updates_per_s": n * steps / (total * 1e-3),
            "mid_beat_1000_steps": {"first_step": chunk * (len(ms) // 2), "ms_per_step": mid / chunk,
                                    "cell_updates_per_s": n * chunk / (mid * 1e-3)},
            "activated_fraction": float(np.isfinite(act).mean()), "state_finite": finite}


def run_sweep(ctx, args, stream, torch):
    """Batched parametric sweep: args.sweep_jobs slab jobs drawn from the
    configured distribution (sizes log-uniform 50k-2M tets, G_Ks / G_Kr
    scalings U[0.5, 1.5], p = 0.5 ischemic sphere with [K]o = 8 mM), all
    advanced together -- one node launch + one cell launch per step for the
    whole batch, captured-graph replay -- against the same jobs stepped one
    job at a time."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2112_12854_b300 import ep
    specs = w.sweep_jobs(n_jobs=256)[:args.sweep_jobs]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=8) as pool:
        plans = list(pool.map(lambda sp: ep.plan_from_case(w.slab_from_spec(sp)), specs))
    jobs = [ep.Job(ctx, plan=p) for p in plans]
    for p in plans:
        p.destroy()
    build_s = time.perf_counter() - t0
    cells = sum(j.n_cells for j in jobs)
    chosen, _ = ep.autotune(jobs, 2)
    ep.step(jobs, 5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ep.step(jobs, args.sweep_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / args.sweep_steps
    for j in jobs:                       # build each job's own plan and graph outside the timing
        j.step(64)
    torch.cuda.synchronize()
    e0.record(stream)
    for j in jobs:
        j.step(args.sweep_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_u = e0.elapsed_time(e1) / args.sweep_steps
    small = [j for j in jobs if j.n_cells < 200_000]
    out = {"jobs": len(jobs), "configured_jobs": 256, "cells": cells, "steps": args.sweep_steps,
           "batched_ms_per_step": ms_b, "batched_cell_updates_per_s": cells / (ms_b * 1e-3),
           "one_job_at_a_time_ms_per_step": ms_u, "one_job_at_a_time_cell_updates_per_s": cells / (ms_u * 1e-3),
           "cell_variant": int(chosen[0]), "host_build_s": build_s}
    if small:
        sc = sum(j.n_cells for j in small)
        ep.step(small, 64)                # the small batch's own plan and graph, outside the timing
        torch.cuda.synchronize()
        e0.record(stream)
        ep.step(small, args.sweep_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        msb = e0.elapsed_time(e1) / args.sweep_steps
        e0.record(stream)
        for j in small:
            j.step(args.sweep_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        msu = e0.elapsed_time(e1) / args.sweep_steps
        out["small_jobs"] = {"jobs": len(small), "cells": sc, "batched_cell_updates_per_s": sc / (msb * 1e-3),
                             "one_job_at_a_time_cell_updates_per_s": sc / (msu * 1e-3)}
    for j in jobs:
        j.destroy()
    return out


def run_heart(ctx, args, stream, torch):
    """Synthetic whole heart with its conduction system at full scale: about
    9.3M tets (ventricles TP06, atria Courtemanche) and a 50k-node graph
    (atrial bundle, AV delay line, two Purkinje trees with 2000 resistive
    PMJs, triggered atrial communication nodes); FP32 mixed, dt 0.02 ms."""
    from paper_2112_12854_b300 import ep
    case, g = w.whole_heart(h=0.4, scale=1.0, n_tree=50_000)
    node_model = np.array([ps.model for ps in case.param_sets], np.uint8)[g.param_set]
    job = ep.job_from_case(ctx, case)
    job.attach_graph(g, node_model=node_model)
    gi = job.graph_info()
    ep.autotune([job], 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    modes = {}
    # the graph's diffusion substeps: one launch per substep, then all substeps in one launch
    # (the library default); the same steps, bitwise the same results
    for name, mode in (("launch_per_substep", ep.EP_GRAPH_SUBSTEPS_LAUNCHES),
                       ("one_launch", ep.EP_GRAPH_SUBSTEPS_LOCAL)):
        ctx.set_graph_kernel(mode)
        job.step(5)
        torch.cuda.synchronize()
        e0.record(stream)
        job.step(args.heart_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.heart_steps
        node_graph_ms, cell_ms = ep.time_kernels([job], 20)
        modes[name] = {"ms_per_step": ms, "node_and_graph_kernels_ms": node_graph_ms, "cell_kernel_ms": cell_ms}
    job.destroy()
    ms = modes["one_launch"]["ms_per_step"]
    return {"cells": case.n_cells, "graph_nodes": gi["n_nodes"], "junctions": gi["n_junctions"],
            "graph_substeps": gi["substeps"], "steps": args.heart_steps, "ms_per_step": ms,
            "cell_updates_per_s": case.n_cells / (ms * 1e-3),
            "node_and_graph_kernels_ms": modes["one_launch"]["node_and_graph_kernels_ms"],
            "cell_kernel_ms": modes["one_launch"]["cell_kernel_ms"], "graph_substep_modes": modes}


def run_bidomain(ctx, args, dims, stream, torch, peak):
    """Bidomain on the benchmark wedge (Eq. 1, Eqs. 5-6): the ventricular
    conductivities of Table 2 (intracellular 0.17 / 0.019, extracellular
    0.62 / 0.24 mS/mm over chi C_m = 1.4 uF/mm^3), FP32 mixed, the
    library's default solver (restarted GMRES(12), stopping rule). Timed after
    args.bido_warmup steps, once the stimulated front is moving; the
    elliptic-solve kernel is placed against HBM with its own algorithmic
    byte count."""
    from paper_2112_12854_b300 import ep
    case = wedge_case(dims)
    for ps in case.param_sets:
        ps.D_l, ps.D_t = 0.17 / 1.4, 0.019 / 1.4
    job = ep.job_from_case(ctx, case)
    job.enable_bidomain(0.62 / 1.4, 0.24 / 1.4)
    job.step(args.bido_warmup)
    torch.cuda.synchronize()
    st0 = job.bidomain_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    job.step(args.bido_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.bido_steps
    st1 = job.bidomain_stats()
    node_ms, cell_ms = ep.time_kernels([job], 3)
    job.destroy()
    solve_ms = ms - node_ms - cell_ms
    iters = (st1["total_iters"] - st0["total_iters"]) / args.bido_steps
    gbs = (st1["alg_bytes"] - st0["alg_bytes"]) / args.bido_steps / (solve_ms * 1e-3) / 1e9
    return {"cells": case.n_cells, "steps": args.bido_steps, "warmup_steps": args.bido_warmup,
            "ms_per_step": ms, "cell_updates_per_s": case.n_cells / (ms * 1e-3),
            "arnoldi_steps_per_step": iters, "solve_ms_per_step": solve_ms,
            "node_kernel_ms": node_ms, "cell_kernel_ms": cell_ms,
            "solve_phase_ms_per_step": {k: (b - a) / args.bido_steps for k, a, b in
                                        zip(("node_values", "fluxes_and_dots", "gs_pass2", "gs_pass3", "updates"),
                                            st0["phase_ms"], st1["phase_ms"])},
            "solver": "restarted GMRES(12), classical Gram-Schmidt, started from 2 v_e^n - v_e^(n-1), "
                      "tol 1e-5 relative / 1e-3 mV/ms per cell absolute",
            "solve_roofline": {"bound": "hbm", "kernel": "bido_kernel<float>", "achieved": gbs, "peak": peak,
                               "unit": "GB/s", "frac": gbs / peak,
                               "alg_bytes_per_step": (st1["alg_bytes"] - st0["alg_bytes"]) / args.bido_steps},
            "last_rel_res": st1["last_res"] / max(st1["last_bnorm"], 1e-300), "failed": st1["failed"]}


def run_serving(ctx, args, capacity_cups, rank, world, dist):
    """Two serving runs of the job-stream workload (sizes log-uniform 20k-4M
    cells, 100-800 ms simulated, 70 % slabs / 30 % whole-heart topology at
    1/4 scale, Poisson arrivals). First at the configured args.serve_rate
    jobs/s, which offers about 3.4e11 cell-updates/s, an order of magnitude
    above one B300's capacity, so it runs overloaded by construction and is
    cut off at a time limit; the cell-updates/s the GPU executed there,
    saturated by this job mix, is the serving capacity. Then at
    args.serve_load x that capacity, where latencies are meaningful (without
    the overloaded run, the capacity is the headline step's rate, which the
    mix of smaller and graph-carrying jobs does not reach). Requests are
    sharded across ranks by id."""
    from paper_2112_12854_b300.serving import LibBackend, Server, config5_requests, summarize
    probe = config5_requests(1.0, 400.0, seed=99)           # the job mix, for its mean work per job
    mean_work = float(np.mean([r.n_cells * r.n_steps for r in probe]))
    out = {"headline_capacity_jobs_per_s": capacity_cups / mean_work, "mean_job_cell_updates": mean_work}
    for name in ("configured", "load"):
        if name == "configured":
            key, rate = "configured_%g_per_s" % args.serve_rate, args.serve_rate
            window = limit = args.serve_window_configured
        else:
            sat = out.get("configured_%g_per_s" % args.serve_rate, {}).get("executed_cell_updates_per_s")
            cap_cups = sat / world if sat else capacity_cups
            cap_jobs = cap_cups / mean_work
            out["capacity_jobs_per_s"] = cap_jobs
            out["capacity_source"] = ("cell-updates/s executed by the overloaded run (this job mix, saturated)"
                                      if sat else "the headline step's cell-updates/s")
            key, rate = "load_%.2f" % args.serve_load, args.serve_load * cap_jobs * world
            window, limit = args.serve_window, args.serve_window + 90.0
        if window <= 0:
            continue
        reqs = config5_requests(rate, window, seed=1 if name == "configured" else 0)
        srv = Server(LibBackend(ctx), steps_per_iter=250, workers=4, rank=rank, world=world)
        t0 = time.perf_counter()
        res = srv.run(reqs, time_limit=limit)
        wall = time.perf_counter() - t0
        if dist is not None:
            allr = [None] * world
            dist.all_gather_object(allr, [(r.latency, r.n_cells * r.n_steps, r.error) for r in res])
            flat = [x for part in allr for x in part]
            lat = np.array([x[0] for x in flat if x[2] is None])
            work = sum(x[1] for x in flat if x[2] is None)
            summ = {"completed": len(lat), "cell_updates_per_s": work / wall,
                    "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
                    "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None}
        else:
            summ = summarize(res, wall, srv.log, srv.unfinished_ages)
        summ.update({"offered_jobs_per_s": rate, "arrivals": len(reqs), "window_s": window,
                     "time_limit_s": limit, "wall_s": wall, "unfinished": len(srv.unfinished) * world,
                     "max_resident": max((x["resident"] for x in srv.log), default=0)})
        if dist is not None:
            summ["executed_cell_updates_per_s"] = summ["cell_updates_per_s"]
        out[key] = summ
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--tune-steps", type=int, default=5, help="steps per cell-kernel variant in the autotuner")
    ap.add_argument("--cell-variant", type=int, default=-1,
                    help="FP32 cell-kernel launch shape (0..7) instead of the autotuner's choice")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--small", action="store_true", help="debug: 1/8-volume crop instead of the full wedge")
    ap.add_argument("--heart-steps", type=int, default=200, help="timed steps of the whole-heart leg (0 = skip)")
    ap.add_argument("--beat-steps", type=int, default=20000,
                    help="steps of the whole-beat leg on the headline workload (400 ms; 0 = skip)")
    ap.add_argument("--sweep-jobs", type=int, default=256, help="jobs of the batched parametric sweep (0 = skip; "
                    "the configured sweep has 256)")
    ap.add_argument("--sweep-steps", type=int, default=200)
    ap.add_argument("--bido-steps", type=int, default=100, help="timed steps of the bidomain leg (0 = skip)")
    ap.add_argument("--bido-warmup", type=int, default=100)
    ap.add_argument("--serve-window", type=float, default=780.0,
                    help="seconds of Poisson arrivals in the serving run at --serve-load x capacity (0 = no serving "
                         "leg at all); at 0.7 x capacity 780 s gives about 300 completions")
    ap.add_argument("--serve-window-configured", type=float, default=60.0,
                    help="seconds of arrivals at the configured rate (overloaded; cut off at the same time)")
    ap.add_argument("--serve-load", type=float, default=0.7, help="offered load of the first serving run, "
                    "as a fraction of the measured capacity")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="arrival rate of the configured (overloaded) run")
    ap.add_argument("--time-budget", type=float, default=1500.0,
                    help="seconds after which the optional legs (sweep, bidomain, heart, serving) are skipped")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    t_start = time.perf_counter()
    skipped = []

    def budget_left(leg, needs_s):
        """True if the leg (about needs_s seconds) fits the time budget; else it is skipped."""
        if time.perf_counter() - t_start + needs_s <= args.time_budget:
            return True
        skipped.append(leg)
        return False
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2112_12854_b300 import ep
    dims = dict(nx=100, ny=100, nz=20, h=0.25) if args.small else WEDGE
    case = wedge_case(dims)
    N = case.n_cells
    ctx = ep.Context()
    alu = ep.alu_peaks(ctx)
    job = ep.job_from_case(ctx, case, precision=ep.EP_FP32_MIXED)
    info = job.info()
    stream = torch.cuda.current_stream()
    # the job's initial state on the host, as the e2e leg uploads it: the variables the FP32 job
    # stores in FP32 as float32 (exact), the compensated concentrations as float64
    nvar = len(ep.model_varnames(ep.EP_TP06))
    comp = ep.model_var_compensated(ep.EP_TP06)
    host_state = [torch.empty(N, dtype=torch.float64 if comp[v] else torch.float32, pin_memory=True).numpy()
                  for v in range(nvar)]
    for v in range(nvar):
        if comp[v]:
            job.read(v, out=host_state[v])
        else:
            job.read_f32(v, out=host_state[v])

    # warm-up (the autotuner's steps are part of it), then the timed region: K steps
    # (captured-graph replay) bracketed by barrier + sync
    if args.cell_variant >= 0:
        ep.set_cell_variant(ctx, ep.EP_FP32_MIXED, args.cell_variant)
        chosen, variant_ms = np.array([args.cell_variant, -1]), None
    else:
        chosen, variant_ms = ep.autotune([job], args.tune_steps)
    job.step(args.warmup)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    job.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * N * args.steps / (ms * 1e-3)
    finite = job.check_finite()

    # per-kernel device time (CUDA events on the launching stream, direct launches)
    node_ms, cell_ms = ep.time_kernels([job], min(args.steps, 200))
    peak, peak_kind = measured_peaks()
    incid = 4.0 * N
    iw = info["index_width"]
    cell_b = cell_bytes(iw)
    cell_gbs = cell_b * N / (cell_ms * 1e-3) / 1e9
    niw = info["node_index_width"]
    node_bytes = node_bytes_per_incidence(niw) * incid + 4.0 * info["n_nodes"]
    traffic = traffic_from_profile(N)
    step_s = ms / args.steps * 1e-3
    roofline = {"bound": "hbm", "kernel": "cell_kernel<float>", "achieved": cell_gbs, "peak": peak,
                "unit": "GB/s", "frac": cell_gbs / peak, "traffic": traffic,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, copy)" if peak_kind == "measured"
                else "fallback 6.4 TB/s",
                "algorithmic_bytes_per_cell": cell_b, "index_width": iw, "node_index_width": niw,
                "cell_kernel_ms": cell_ms, "node_kernel_ms": node_ms,
                "cell_variant": int(chosen[0]), "autotune_ms": None if variant_ms is None else [round(float(x), 4) for x in variant_ms[0]],
                "node_kernel_gbs": node_bytes / (node_ms * 1e-3) / 1e9,
                "step_gbs": (cell_b * N + node_bytes) / ((cell_ms + node_ms) * 1e-3) / 1e9,
                # the same kernels against the shared-face byte floor (277 B per step, 245 B of it
                # the cell kernel's), the step taken from the timed region
                "shared_face_floor": {"step_bytes_per_cell": FACE_STEP_FLOOR,
                                      "step_frac": FACE_STEP_FLOOR * N / step_s / 1e9 / peak,
                                      "cell_bytes_per_cell": FACE_CELL_FLOOR,
                                      "cell_frac": FACE_CELL_FLOOR * N / (cell_ms * 1e-3) / 1e9 / peak},
                "alu": alu_side(N, cell_ms, alu)}

    # end to end through the public API with host buffers: the initial state uploaded from pinned
    # host memory, K steps, V read back every OUTPUT_EVERY steps, the activation map at the end
    e2e = None
    if not args.no_e2e:
        vout = torch.empty(N, dtype=torch.float32, pin_memory=True).numpy()
        aout = torch.empty(N, dtype=torch.float32, pin_memory=True).numpy()
        job.reset_activation()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        job.step_index = 0
        for v in range(nvar):
            if comp[v]:
                job.write(v, host_state[v])
            else:
                job.write_f32(v, host_state[v])
        done, reads = 0, 0
        while done < args.steps:
            k = min(OUTPUT_EVERY, args.steps - done)
            job.step(k)
            done += k
            job.read_f32(0, out=vout)
            reads += 1
        job.activation_times_f32(out=aout)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        barrier()
        h2d = sum(x.nbytes for x in host_state)
        e2e = {"value": world * N * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": (reads + 1) * 4 * N / args.steps,
               "note": f"state uploaded from pinned host memory (the variables the FP32 job stores in FP32 as "
                       f"float32, its compensated concentrations as float64), V read back every {OUTPUT_EVERY} "
                       "steps, the activation map at the end (float32)"}
    job.destroy()

    # plain FP64 path on the same workload
    job64 = ep.job_from_case(ctx, case, precision=ep.EP_FP64_PLAIN)
    chosen64, _ = ep.autotune([job64], 1)
    job64.step(2)
    torch.cuda.synchronize()
    e0.record(stream)
    job64.step(args.fp64_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    node64_ms, cell64_ms = ep.time_kernels([job64], 2)
    job64.destroy()
    # the plain FP64 cell kernel runs on the FP64 pipe: its roof is the measured FP64 FMA rate;
    # its FP64 flops per cell (2 per DFMA, 1 per DADD / DMUL) come from the ncu summary
    f64_per_cell = profile_value("cell_kernel_fp64_crop.md", "fp64_flops_per_cell")
    f64_peak = alu["fp64_fma_flops"] / 1e12
    f64_ach = None if f64_per_cell is None else f64_per_cell * N / (cell64_ms * 1e-3) / 1e12
    fp64 = {"value": N * args.fp64_steps / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps,
            "steps": args.fp64_steps, "cell_variant": int(chosen64[1]),
            "roofline": {"bound": "alu", "kernel": "cell_kernel<double>", "achieved": f64_ach, "peak": f64_peak,
                         "unit": "TFLOP/s", "frac": None if f64_ach is None else f64_ach / f64_peak,
                         "peak_source": "measured FP64 FMA issue rate (ep_alu_peaks)",
                         "fp64_flops_per_cell": f64_per_cell, "cell_kernel_ms": cell64_ms,
                         "node_kernel_ms": node64_ms}}

    sweep = None
    if args.sweep_jobs > 0 and budget_left("batched_sweep", 240.0):
        sweep = run_sweep(ctx, args, stream, torch)

    bido = None
    if args.bido_steps > 0 and budget_left("bidomain", 60.0):
        bido = run_bidomain(ctx, args, dims, stream, torch, peak)

    beat = None
    if args.beat_steps > 0 and budget_left("beat", 40.0):
        beat = run_beat(ctx, args, dims, stream, torch)

    heart = None
    if args.heart_steps > 0 and budget_left("whole_heart", 90.0):
        heart = run_heart(ctx, args, stream, torch)

    serving = None
    if args.serve_window > 0 and budget_left("serving", args.serve_window + args.serve_window_configured + 200.0):
        serving = run_serving(ctx, args, value / world, rank, world, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, st, cells, cores = oracle_throughput(CROP, args.cpu_budget)
        import oracle
        prev = oracle.set_threads(1)
        val1, st1, _, _ = oracle_throughput(CROP, args.cpu_budget / 3)
        oracle.set_threads(prev)
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"oracle on a {CROP['nx']}x{CROP['ny']}x{CROP['nz']}-cube crop of the wedge "
                         f"({cells} cells), {st} steps",
               "value_1core": val1, "sample_1core": f"the same crop on one thread, {st1} steps"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"ventricular wedge slab {dims['nx']}x{dims['ny']}x{dims['nz']} cubes "
                                      f"of {dims['h']} mm x 6 tets, TP06 endo/M/epi, fibres -60..+60 deg",
                          "cells": N, "nodes": info["n_nodes"], "dt_ms": case.dt,
                          "precision": "FP32 with two-float compensated [Na]i/[K]i/[Ca]SR accumulation",
                          "l2": f"inputs larger than L2 ({info['device_bytes'] / 1e9:.2f} GB resident, "
                                f"~{(cell_b * N + node_bytes) / 1e9:.2f} GB moved per step > 126 MB)",
                          "index_width": iw,
                          "parallelism": f"replicas x{world}", "graph_replay": True},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": (1 if int(chosen[0]) in FUSED_VARIANTS else 2) * args.steps, "fp64_plain": fp64,
               "alu_peaks": {"fp32_fma_tflops": alu["fp32_fma_flops"] / 1e12,
                             "mufu_ex2_tops": alu["mufu_ex2_ops"] / 1e12,
                             "fp64_fma_tflops": alu["fp64_fma_flops"] / 1e12,
                             "source": "ep_alu_peaks: independent FMA / ex2 chains on every SM, CUDA events"},
               "speedup_vs_fp64_plain": value / world / fp64["value"], "state_finite": finite,
               "beat": beat, "batched_sweep": sweep, "bidomain": bido, "whole_heart": heart, "serving": serving,
               "legs_skipped_for_time": skipped, "bench_wall_s": time.perf_counter() - t_start}
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
