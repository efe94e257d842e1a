"""Continuous-batching serving loop for simulation jobs.

Requests (a mesh + parameters + a number of time steps) arrive over time.
The server
  - prepares each arrived request on worker threads: mesh generation and the
    host-only planner (ep_plan_create), which touch no device;
  - admits prepared jobs in arrival order while their device bytes (exact,
    from the plan) fit the free device memory, and uploads them
    (ep_job_create, on a private stream that does not wait for queued steps);
  - advances every resident job together: one ep_step call per iteration,
    i.e. one node launch + one cell launch per time step for the whole
    resident set, replayed from a captured CUDA graph while the set is
    unchanged. Jobs admitted while others run join at the next iteration
    (continuous batching); each iteration takes at most ``steps_per_iter``
    steps and never more than the resident job closest to completion needs,
    so no job overshoots its duration;
  - retires a job when it has taken its steps: V and the activation map are
    read back to host, the device memory is released, and the completion
    latency (finish - arrival, queueing included) is recorded.
The host may run at most ``max_inflight`` iterations ahead of the GPU.

The backend interface is explicit so that the scheduling logic can be tested
without a GPU (see tests/test_serving_host.py).
"""
from __future__ import annotations

import math
import time
from concurrent.futures import ThreadPoolExecutor
from concurrent.futures import wait as wait_futures
from dataclasses import dataclass, field
from typing import Any, Callable

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float                     # seconds after the server starts
    n_steps: int
    prepare: Callable[[], Any]         # host-only: returns a backend token (a plan)
    n_cells: int = 0
    keep_result: bool = True
    meta: dict = field(default_factory=dict)


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    n_cells: int
    n_steps: int
    V: np.ndarray | None = None
    act: np.ndarray | None = None
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class LibBackend:
    """Backend over the C ABI (paper_2112_12854_b300.ep) and torch."""

    def __init__(self, ctx, *, reserve_bytes: int = 2 << 30, budget_bytes: int | None = None):
        import torch
        from . import ep
        self.ep, self.torch, self.ctx = ep, torch, ctx
        self.reserve = reserve_bytes
        self.budget = budget_bytes
        self.resident_bytes = 0
        self._bytes: dict[int, int] = {}

    def bytes_of(self, plan) -> int:
        return int(plan.device_bytes)

    def n_cells(self, plan) -> int:
        return int(plan.n_cells)

    def free_bytes(self) -> int:
        if self.budget is not None:
            return self.budget - self.resident_bytes
        free, _ = self.torch.cuda.mem_get_info()
        cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        return free + cached - self.reserve

    def create(self, plan):
        job = self.ep.Job(self.ctx, plan=plan)
        self._bytes[id(job)] = int(plan.device_bytes)
        self.resident_bytes += int(plan.device_bytes)
        plan.destroy()
        return job

    def step(self, jobs, k: int):
        self.ep.step(jobs, k)

    def mark(self):
        ev = self.torch.cuda.Event()
        ev.record(self.ctx.stream)
        return ev

    def wait(self, mark):
        mark.synchronize()

    def healthy(self, job) -> bool:
        return job.check_finite()

    def finish(self, job, keep: bool):
        V = job.V if keep else None
        act = job.activation_times() if keep else None
        job.destroy()
        self.resident_bytes -= self._bytes.pop(id(job), 0)
        return V, act


class Server:
    def __init__(self, backend, *, steps_per_iter: int = 250, max_resident: int = 256, workers: int = 4,
                 max_prepared: int | None = None, max_inflight: int = 2, clock=time.perf_counter,
                 sleep=time.sleep, rank: int = 0, world: int = 1):
        self.b = backend
        self.steps_per_iter = steps_per_iter
        self.max_resident = max_resident
        self.workers = workers
        self.max_prepared = max_prepared if max_prepared is not None else 2 * workers
        self.max_inflight = max_inflight
        self.clock, self.sleep = clock, sleep
        self.rank, self.world = rank, world
        self.log: list[dict] = []
        self.unfinished: list[int] = []
        self.unfinished_ages: list[float] = []
        self.cut_s: float | None = None
        self.cancelled: set[int] = set()

    def cancel(self, rid: int):
        """Cancel a request: dropped if not yet admitted, released (no
        result) at the next iteration boundary if resident."""
        self.cancelled.add(rid)

    def run(self, requests: list[Request], *, time_limit: float | None = None) -> list[Result]:
        """Serve the requests (those with rid % world == rank); returns the
        results of completed jobs, in completion order."""
        reqs = sorted((r for r in requests if r.rid % self.world == self.rank), key=lambda r: (r.arrival, r.rid))
        pending = list(reversed(reqs))            # pop() gives the earliest
        queue: list[Request] = []                  # arrived, not yet preparing
        preparing: list[tuple[Request, Any]] = []  # (request, future), arrival order
        ready: list[tuple[Request, Any]] = []      # (request, token), arrival order
        resident: list[list] = []                  # [request, job, remaining, admitted]
        inflight: list[Any] = []
        results: list[Result] = []
        pool = ThreadPoolExecutor(max_workers=self.workers)
        t0 = self.clock()
        try:
            while pending or queue or preparing or ready or resident:
                now = self.clock() - t0
                if time_limit is not None and now > time_limit:
                    break
                while pending and pending[-1].arrival <= now:
                    queue.append(pending.pop())
                if self.cancelled:
                    for r in [r for r in queue if r.rid in self.cancelled] + \
                             [r for r, _ in ready if r.rid in self.cancelled]:
                        results.append(Result(r.rid, r.arrival, now, now, r.n_cells, r.n_steps, error="cancelled"))
                    queue = [r for r in queue if r.rid not in self.cancelled]
                    ready = [(r, t) for r, t in ready if r.rid not in self.cancelled]
                    keep = []
                    for x in resident:
                        if x[0].rid in self.cancelled:
                            self.b.finish(x[1], False)
                            results.append(Result(x[0].rid, x[0].arrival, x[3], now, x[0].n_cells, x[0].n_steps,
                                                  error="cancelled"))
                        else:
                            keep.append(x)
                    resident = keep
                while queue and len(preparing) + len(ready) < self.max_prepared:
                    r = queue.pop(0)
                    preparing.append((r, pool.submit(r.prepare)))
                # collect finished preparations in arrival order
                while preparing and preparing[0][1].done():
                    r, fut = preparing.pop(0)
                    try:
                        ready.append((r, fut.result()))
                    except Exception as exc:   # a request that cannot be planned fails alone
                        results.append(Result(r.rid, r.arrival, now, now, r.n_cells, r.n_steps, error=str(exc)))
                # admission by device memory, arrival order
                while ready and len(resident) < self.max_resident:
                    r, tok = ready[0]
                    need = self.b.bytes_of(tok)
                    if need > self.b.free_bytes():
                        if resident:
                            break                  # wait for a retirement to free memory
                        ready.pop(0)
                        results.append(Result(r.rid, r.arrival, now, now, r.n_cells, r.n_steps,
                                              error=f"needs {need} device bytes, more than the device offers"))
                        continue
                    ready.pop(0)
                    job = self.b.create(tok)
                    resident.append([r, job, r.n_steps, self.clock() - t0])
                if not resident:
                    if preparing:
                        wait_futures([preparing[0][1]])   # block until the oldest preparation ends
                    elif pending and not queue and not ready:
                        self.sleep(max(0.0, min(pending[-1].arrival - (self.clock() - t0), 0.05)))
                    continue
                k = min(self.steps_per_iter, min(x[2] for x in resident))
                self.b.step([x[1] for x in resident], k)
                inflight.append(self.b.mark())
                self.log.append({"t": self.clock() - t0, "resident": len(resident), "steps": k,
                                 "cells": sum(x[0].n_cells for x in resident)})
                if len(inflight) > self.max_inflight:
                    self.b.wait(inflight.pop(0))
                for x in resident:
                    x[2] -= k
                done = [x for x in resident if x[2] == 0]
                if done:
                    resident = [x for x in resident if x[2] > 0]
                    for r, job, _, adm in done:
                        err = None if self.b.healthy(job) else "non-finite state"
                        V, act = self.b.finish(job, r.keep_result and err is None)
                        results.append(Result(r.rid, r.arrival, adm, self.clock() - t0, r.n_cells, r.n_steps,
                                              V=V, act=act, error=err))
                    inflight.clear()               # finish() synchronised the stream
        finally:
            t_cut = self.clock() - t0
            pool.shutdown(wait=True, cancel_futures=True)
            for r, job, _, _ in resident:          # stopped by the time limit: release, no result
                self.b.finish(job, False)
            self.unfinished = [x[0].rid for x in resident] + [r.rid for r, _ in ready] + \
                              [r.rid for r, _ in preparing] + [r.rid for r in queue] + [r.rid for r in pending]
            # age at the cut-off of every job that had arrived but not finished: a lower bound
            # of its latency (the latency distribution is censored there)
            arrived = [x[0] for x in resident] + [r for r, _ in ready] + [r for r, _ in preparing] + queue
            self.unfinished_ages = [t_cut - r.arrival for r in arrived]
            self.cut_s = t_cut
        return results


def summarize(results: list[Result], wall_s: float, log: list[dict] | None = None,
              unfinished_ages: list[float] | None = None) -> dict:
    """Completed-job throughput and latency percentiles; with the server log,
    also the cell-updates/s the GPU executed (unfinished jobs included). With
    the ages at the cut-off of the jobs that had arrived but not finished,
    also the percentiles over every arrived job, each unfinished one counted
    at its age: lower bounds of the true percentiles when the run was cut
    off (a censored sample)."""
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
    work = float(sum(r.n_cells * r.n_steps for r in ok))
    out = {"completed": len(ok), "failed": len(results) - len(ok),
           "cell_updates_per_s": work / wall_s if wall_s > 0 else 0.0,
           "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
           "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
           "mean_latency_s": float(lat.mean()) if len(lat) else None,
           "executed_cell_updates_per_s": (sum(x["steps"] * x["cells"] for x in log) / wall_s
                                           if log and wall_s > 0 else None),
           "errors": sorted({r.error for r in results if r.error})[:3]}
    if unfinished_ages is not None:
        allv = np.concatenate([lat, np.asarray(unfinished_ages, float)])
        out["censored"] = {"arrived_unfinished": len(unfinished_ages),
                           "p50_latency_lower_bound_s": float(np.percentile(allv, 50)) if len(allv) else None,
                           "p99_latency_lower_bound_s": float(np.percentile(allv, 99)) if len(allv) else None,
                           "max_age_at_cutoff_s": float(max(unfinished_ages)) if unfinished_ages else None}
    return out


def poisson_arrivals(rate_per_s: float, duration_s: float, rng) -> np.ndarray:
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s:
            return np.array(out)
        out.append(t)


def log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def config5_requests(rate_per_s: float, window_s: float, *, seed: int = 0, n_min: int = 20_000,
                     n_max: int = 4_000_000, dur_ms=(100.0, 800.0), heart_fraction: float = 0.3,
                     dt: float = 0.02, keep_result: bool = False) -> list[Request]:
    """The serving workload: Poisson arrivals at rate_per_s over window_s
    seconds; sizes log-uniform in [n_min, n_max] cells; simulated durations
    uniform in dur_ms; 70 % ventricular slabs (nx = ny = 5 nz cubes of
    0.25 mm, TP06, corner stimulus) and 30 % whole-heart-topology meshes at
    1/4 scale resized to the drawn size. Meshes and plans are built lazily
    on the server's worker threads."""
    import workloads as w
    from . import ep
    rng = np.random.default_rng(w.MASTER_SEED + 5 + seed)
    times = poisson_arrivals(rate_per_s, window_s, rng)
    reqs = []
    for rid, t in enumerate(times):
        n = int(log_uniform(rng, n_min, n_max))
        dur = float(rng.uniform(*dur_ms))
        heart = rng.uniform() < heart_fraction
        if heart:
            h = w.heart_h_for_cells(n, 0.25)
            # explicit stability: the diffusion operator's spectral radius grows like 1/h^2, so a
            # finer voxel takes a proportionally smaller step (dt = 0.02 ms is stable down to h = 0.25 mm)
            jdt = min(dt, dt * (h / 0.25) ** 2)

            def prep(h=h, jdt=jdt):
                return ep.plan_from_case(w.heart_case(h=h, scale=0.25, dt=jdt))
        else:
            jdt = dt
            nz = max(1, int(round((n / 150.0) ** (1.0 / 3.0))))
            spec = dict(nx=5 * nz, ny=5 * nz, nz=nz, h=0.25, gks=1.0, gkr=1.0, ischemic=False, radius=0.0,
                        centre=[0.0, 0.0, 0.0])

            def prep(spec=spec):
                return ep.plan_from_case(w.slab_from_spec(spec, dt=dt))
            n = 6 * 25 * nz ** 3
        steps = int(round(dur / jdt))
        reqs.append(Request(rid=rid, arrival=float(t), n_steps=steps, prepare=prep, n_cells=n,
                            keep_result=keep_result,
                            meta={"kind": "heart" if heart else "slab", "dt": jdt, "duration_ms": dur}))
    return reqs
