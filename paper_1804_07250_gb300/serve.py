"""Request loop with continuous batching for sampling jobs.

A request asks for k sweeps of one chain on one domain (an Aztec diamond, a
lozenge hexagon or a six-vertex square with domain-wall boundary) at uniform
or log-normal weights, and gets back the final tiling's hash and height
summary.  Requests arrive over time; worker threads build each job's domain,
thresholds and chain as soon as it arrives; the serving loop admits built jobs
into the running batch whenever the HBM budget allows, advances every admitted
chain together (one work list per launch, graph-captured blocks), and retires
jobs as they finish, so new work overlaps old work on the device.  Each job's
random numbers are keyed by its own stream id, so its result does not depend
on what else was in the batch.

Usage (library): ``Server(ctx, budget_bytes).run(requests)``; ``make_requests``
draws the synthetic request mix.
"""
from __future__ import annotations

import dataclasses
import math
import queue
import threading
import time

import numpy as np
import torch

from . import (Batch, Chain, Context, Domain, sixv_thresholds, thresholds)

LOGNORMAL_SIGMA = 0.5


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    kind: str               # "aztec" | "hexagon" | "dwbc"
    size: tuple
    weights: str            # "uniform" | "lognormal"
    sweeps: int
    seed: int


@dataclasses.dataclass
class Job:
    req: Request
    chain: Chain = None
    sites: int = 0
    footprint: int = 0
    remaining: int = 0
    admitted: float = -1.0
    built: float = -1.0
    done: float = -1.0
    result_hash: int = 0
    keep: object = None


def make_requests(n: int, rate: float, seed: int = 5, *, aztec=(32, 2048), hexagon=(16, 512),
                  dwbc=(32, 1024), sweeps=(1_000, 100_000)) -> list[Request]:
    """Poisson arrivals at `rate` per second; a third each of Aztec diamonds,
    hexagons (independent sides) and domain-wall six-vertex squares; uniform
    or log-normal weights with equal probability; sweeps log-uniform."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        kind = ("aztec", "hexagon", "dwbc")[int(rng.integers(0, 3))]
        if kind == "aztec":
            size = (int(rng.integers(aztec[0], aztec[1] + 1)),)
        elif kind == "hexagon":
            size = tuple(int(v) for v in rng.integers(hexagon[0], hexagon[1] + 1, size=3))
        else:
            size = (int(rng.integers(dwbc[0], dwbc[1] + 1)),)
        weights = "lognormal" if rng.random() < 0.5 else "uniform"
        k = int(round(math.exp(rng.uniform(math.log(sweeps[0]), math.log(sweeps[1])))))
        out.append(Request(i, float(t[i]), kind, size, weights, k, seed))
    return out


def footprint(dom: Domain, site_thresholds: bool) -> int:
    """Device bytes a job holds while admitted: state, start copy, the
    batch's second buffer, staging and (per-site weights) threshold planes."""
    info = dom.info
    b = 3 * info.packed_bytes + info.canon_bytes + 4 * info.height_count
    if site_thresholds:
        npar = 3 if info.lattice == 1 else 2
        b += info.packed_bytes * 32 * npar // (npar * info.planes) + 4 * info.site_box
    return int(b)


def build_job(ctx: Context, req: Request, stream) -> Job:
    """Domain, thresholds and chain of one request (stream id = request id)."""
    if req.kind == "aztec":
        dom = Domain.aztec(*req.size)
    elif req.kind == "hexagon":
        dom = Domain.hexagon(*req.size)
    else:
        dom = Domain.dwbc(*req.size)
    keep = None
    site = False
    if req.kind == "dwbc":
        if req.weights == "lognormal":
            w6 = np.exp(LOGNORMAL_SIGMA * np.random.default_rng([req.seed, req.rid]).standard_normal(6))
        else:
            w6 = np.ones(6)
        th = thresholds(table16=sixv_thresholds(w6))
    elif req.weights == "lognormal":
        t = torch.empty((dom.info.height, dom.info.width), dtype=torch.int32, device="cuda")
        dom.lognormal_thresholds_device(LOGNORMAL_SIGMA, (req.seed << 32) | req.rid, t, stream=stream)
        stream.synchronize()   # the chain copies the thresholds on another stream
        th = thresholds(site=t)
        keep = t
        site = True
    else:
        th = thresholds(scalar=1 << 31)
    chain = Chain(ctx, dom, seed=req.seed, stream_id=req.rid, th=th)
    return Job(req=req, chain=chain, sites=int(dom.info.sites), footprint=footprint(dom, site),
               remaining=req.sweeps, keep=keep)


class Server:
    """Continuous-batching request loop on one GPU."""

    def __init__(self, ctx: Context, budget_bytes: int, *, block: int = 100, tile_rows: int = 128,
                 sweeps_per_launch: int = 4, workers: int = 2, max_active: int = 4096):
        self.ctx = ctx
        self.budget = budget_bytes
        self.block = block
        self.workers = workers
        self.max_active = max_active
        self.stream = torch.cuda.Stream()
        self.batch = Batch(ctx)
        # membership changes between ticks and worker threads create chains
        # meanwhile: plain launches, no graph capture
        self.batch.set_plan(tile_rows, sweeps_per_launch, -1)

    def run(self, requests: list[Request], *, keep_chains: bool = False):
        """Serve `requests` in real time; returns the finished jobs and stats."""
        todo: "queue.Queue[Request]" = queue.Queue()
        built: "queue.Queue[Job]" = queue.Queue()
        for r in requests:
            todo.put(r)
        t0 = time.perf_counter()

        def worker():
            s = torch.cuda.Stream()
            while True:
                try:
                    r = todo.get_nowait()
                except queue.Empty:
                    return
                wait = r.arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                job = build_job(self.ctx, r, s)
                job.built = time.perf_counter() - t0
                built.put(job)

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for th in threads:
            th.start()
        waiting: list[Job] = []
        active: list[Job] = []
        finished: list[Job] = []
        in_use = 0
        attempts = 0
        busy = 0.0
        peak_active = 0
        peak_in_use = 0
        n = len(requests)
        while len(finished) < n:
            while True:
                try:
                    waiting.append(built.get_nowait())
                except queue.Empty:
                    break
            waiting.sort(key=lambda j: j.req.arrival)
            now = time.perf_counter() - t0
            # admit in arrival order while the budget allows (no overtaking)
            while waiting and len(active) < self.max_active and in_use + waiting[0].footprint <= self.budget:
                j = waiting.pop(0)
                self.batch.add(j.chain)
                j.admitted = now
                in_use += j.footprint
                active.append(j)
            if not active:
                time.sleep(0.0005)
                continue
            peak_active = max(peak_active, len(active))
            peak_in_use = max(peak_in_use, in_use)
            k = min(self.block, min(j.remaining for j in active))
            ts = time.perf_counter()
            self.batch.run(k, stream=self.stream)
            self.stream.synchronize()
            busy += time.perf_counter() - ts
            attempts += k * sum(j.sites for j in active)
            still = []
            for j in active:
                j.remaining -= k
                if j.remaining:
                    still.append(j)
                    continue
                j.result_hash = j.chain.state_hash(stream=self.stream)
                j.done = time.perf_counter() - t0
                self.batch.remove(j.chain)
                in_use -= j.footprint
                if not keep_chains:
                    j.chain.close()
                    j.chain = None
                    j.keep = None
                finished.append(j)
            active = still
        wall = time.perf_counter() - t0
        for th in threads:
            th.join()
        lat = np.array([j.done - j.req.arrival for j in finished])
        stats = {"requests": n, "wall_s": wall, "gpu_busy_s": busy, "attempts": attempts,
                 "attempts_per_s": attempts / wall, "attempts_per_busy_s": attempts / max(busy, 1e-9),
                 "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                 "mean_latency_s": float(lat.mean()), "peak_active": peak_active,
                 "peak_in_use_bytes": peak_in_use}
        return finished, stats


def alone_hash(ctx: Context, req: Request) -> int:
    """The same request run on its own chain, outside any batch."""
    s = torch.cuda.Stream()
    job = build_job(ctx, req, s)
    job.chain.run(req.sweeps, stream=s)
    h = job.chain.state_hash(stream=s)
    job.chain.close()
    return h
