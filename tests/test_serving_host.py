"""Host-side checks of the continuous-batching server (no GPU): a fake
backend records every step so that admission by memory, continuous
batching, exact step counts and rank sharding can be verified."""
import os

import numpy as np
import pytest

from paper_2112_12854_b300.serving import Request, Server, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeJob:
    def __init__(self, tok):
        self.tok = tok
        self.steps = 0


class FakeBackend:
    """Device memory `budget`; each step of a resident set costs
    `cost` seconds per cell-update on the fake clock."""

    def __init__(self, clock, budget, cost=1e-9):
        self.clock, self.budget, self.cost = clock, budget, cost
        self.used = 0
        self.peak = 0
        self.calls = []

    def bytes_of(self, tok):
        return tok["bytes"]

    def free_bytes(self):
        return self.budget - self.used

    def create(self, tok):
        self.used += tok["bytes"]
        self.peak = max(self.peak, self.used)
        return FakeJob(tok)

    def step(self, jobs, k):
        self.calls.append((tuple(j.tok["rid"] for j in jobs), k))
        for j in jobs:
            j.steps += k
        self.clock.t += self.cost * k * sum(j.tok["cells"] for j in jobs)

    def mark(self):
        return None

    def wait(self, m):
        pass

    def healthy(self, job):
        return not job.tok.get("nan", False)

    def finish(self, job, keep):
        self.used -= job.tok["bytes"]
        return (np.full(3, float(job.steps)) if keep else None), None


def _requests(n, rng, arrival_scale=0.01):
    reqs = []
    for rid in range(n):
        cells = int(rng.integers(1000, 50000))
        steps = int(rng.integers(10, 900))
        tok = {"rid": rid, "bytes": cells * 300, "cells": cells}
        reqs.append(Request(rid=rid, arrival=float(rng.uniform(0, n * arrival_scale)), n_steps=steps,
                            prepare=(lambda tok=tok: tok), n_cells=cells))
    return reqs


def test_every_job_takes_exactly_its_steps_and_memory_is_respected():
    rng = np.random.default_rng(0)
    clk = FakeClock()
    be = FakeBackend(clk, budget=40000 * 300 * 3)
    reqs = _requests(40, rng)
    srv = Server(be, steps_per_iter=100, workers=2, clock=clk, sleep=clk.sleep)
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == list(range(40))
    for r in res:
        req = reqs[r.rid]
        assert r.error is None and r.V[0] == req.n_steps          # no overshoot, no shortfall
        assert r.finished >= r.admitted >= r.arrival - 1e-12
    assert be.peak <= be.budget
    # continuous batching: some iterations advance several jobs at once, and the
    # resident set changes between iterations while jobs are still running
    sets = [c[0] for c in be.calls]
    assert max(len(s) for s in sets) > 1
    assert len(set(sets)) > 5
    s = summarize(res, clk.t)
    assert s["completed"] == 40 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_admission_waits_for_memory_and_rejects_oversized():
    clk = FakeClock()
    be = FakeBackend(clk, budget=1000)
    mk = lambda rid, b, arr: Request(rid=rid, arrival=arr, n_steps=50,
                                     prepare=(lambda: {"rid": rid, "bytes": b, "cells": 10}), n_cells=10)
    reqs = [mk(0, 600, 0.0), mk(1, 600, 0.0), mk(2, 5000, 0.0), mk(3, 300, 0.0)]
    res = {r.rid: r for r in Server(be, steps_per_iter=10, clock=clk, sleep=clk.sleep).run(reqs)}
    assert res[2].error and "device bytes" in res[2].error
    assert res[0].error is None and res[1].error is None and res[3].error is None
    # job 1 could only be admitted after job 0 retired (600 + 600 > 1000); arrival order is kept
    assert res[1].admitted >= res[0].finished
    assert be.peak <= 1000


def test_time_limit_releases_resident_jobs():
    clk = FakeClock()
    be = FakeBackend(clk, budget=10 ** 9, cost=1e-6)
    reqs = _requests(10, np.random.default_rng(1))
    srv = Server(be, steps_per_iter=50, clock=clk, sleep=clk.sleep)
    res = srv.run(reqs, time_limit=0.05)
    assert be.used == 0
    assert len(res) + len(srv.unfinished) == 10


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    clk = FakeClock()
    be = FakeBackend(clk, budget=10 ** 9)
    reqs = _requests(23, np.random.default_rng(7))
    res = Server(be, clock=clk, sleep=clk.sleep, rank=rank, world=world).run(reqs)
    got = [None] * world
    dist.all_gather_object(got, sorted(r.rid for r in res))
    if rank == 0:
        out.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_jobs_shard_across_ranks_gloo():
    """Under several ranks each job is served by exactly one rank; the only
    collective is the results gather (no data-path exchange)."""
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = set(got[0]), set(got[1])
    assert not (a & b) and a | b == set(range(23))
    assert all(x % 2 == 0 for x in a) and all(x % 2 == 1 for x in b)


def test_cancel_and_nonfinite_jobs_fail_alone():
    clk = FakeClock()
    be = FakeBackend(clk, budget=10 ** 9)
    reqs = _requests(12, np.random.default_rng(3))
    reqs[4].prepare = (lambda tok={"rid": 4, "bytes": 1000, "cells": 1000, "nan": True}: tok)
    srv = Server(be, steps_per_iter=50, clock=clk, sleep=clk.sleep)
    srv.cancel(7)
    res = {r.rid: r for r in srv.run(reqs)}
    assert res[7].error == "cancelled" and res[4].error == "non-finite state"
    assert all(res[k].error is None for k in res if k not in (4, 7))
    assert be.used == 0
