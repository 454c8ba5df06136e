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
    status: str = "ok"          # "ok" | "cancelled" | "failed: <reason>"
    tail: object = None         # CUDA event of the job's last sweeps run on their own


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
    """Continuous-batching request loop on one GPU.

    Admission: built jobs are admitted oldest first while the HBM budget
    allows; a job that does not fit may be overtaken by later ones that do,
    until it has waited `overtake_s` seconds, after which nothing younger is
    admitted before it.  Ticks: every admitted chain advances `block` sweeps
    per tick; a job with fewer sweeps left leaves the batch and finishes them
    on its own chain on a side stream (its random numbers are keyed by its
    own stream id and sweep index, so the result is the same), so one nearly
    finished job never shortens everybody's tick.  The host waits for the GPU
    only when the batch's membership changes.  Faults handled on the host: a
    request cancelled (``cancel``) leaves at the next tick boundary; a job
    whose domain, thresholds or chain cannot be built (``build_fault`` test
    hook, or a library error) is reported failed; other jobs are unaffected.
    """

    def __init__(self, ctx: Context, budget_bytes: int, *, block: int = 100, tile_rows: int = 128,
                 sweeps_per_launch: int = 4, workers: int = 2, max_active: int = 4096,
                 overtake_s: float = 2.0, build_fault=None):
        self.ctx = ctx
        self.budget = budget_bytes
        self.block = block
        self.workers = workers
        self.max_active = max_active
        self.overtake_s = overtake_s
        self.build_fault = build_fault      # test hook: f(request) -> exception to raise, or None
        self.stream = torch.cuda.Stream()
        self.side = torch.cuda.Stream()
        self.batch = Batch(ctx)
        # membership changes between ticks and worker threads create chains
        # meanwhile: plain launches, no graph capture
        self.batch.set_plan(tile_rows, sweeps_per_launch, -1)
        self._cancel = set()
        self._lock = threading.Lock()

    def cancel(self, rid: int):
        """Ask for request `rid` to be dropped (at the next tick boundary)."""
        with self._lock:
            self._cancel.add(rid)

    def _cancelled(self, rid: int) -> bool:
        with self._lock:
            return rid in self._cancel

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
                try:
                    fault = self.build_fault(r) if self.build_fault else None
                    if fault is not None:
                        raise fault
                    job = build_job(self.ctx, r, s)
                except Exception as e:          # the request fails; the loop goes on
                    job = Job(req=r, status="failed: %s" % e)
                job.built = time.perf_counter() - t0
                built.put(job)

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for th in threads:
            th.start()
        waiting: list[Job] = []
        active: list[Job] = []
        tails: list[Job] = []          # finishing alone on the side stream
        finished: list[Job] = []
        in_use = 0
        attempts = 0
        busy = 0.0
        peak_active = 0
        peak_in_use = 0
        ticks = 0
        inflight = False               # a tick enqueued without waiting for it
        n = len(requests)

        def settle():
            # the batch's membership changes only with no tick in flight
            nonlocal inflight
            if inflight:
                self.stream.synchronize()
                inflight = False

        def release(j, status=None):
            nonlocal in_use
            if status:
                j.status = status
            in_use -= j.footprint
            if not keep_chains and j.chain is not None:
                j.chain.close()
                j.chain = None
                j.keep = None
            j.done = time.perf_counter() - t0
            finished.append(j)

        while len(finished) < n:
            while True:
                try:
                    j = built.get_nowait()
                except queue.Empty:
                    break
                if j.chain is None:                     # failed to build
                    j.done = time.perf_counter() - t0
                    finished.append(j)
                else:
                    waiting.append(j)
            now = time.perf_counter() - t0
            # cancelled requests leave between ticks
            for lst in (waiting, active):
                for j in [j for j in lst if self._cancelled(j.req.rid)]:
                    lst.remove(j)
                    if lst is active:
                        settle()
                        self.batch.remove(j.chain)
                    in_use += 0 if lst is active else j.footprint   # waiting jobs hold nothing yet
                    release(j, "cancelled")
            # jobs finishing alone: done when their event has completed
            for j in [j for j in tails if j.tail.query()]:
                tails.remove(j)
                j.result_hash = j.chain.state_hash(stream=self.side)
                release(j)
            # admission: oldest first, overtaking a job that does not fit only
            # until it has waited overtake_s
            waiting.sort(key=lambda j: j.req.arrival)
            blocked = False
            for j in list(waiting):
                if len(active) + len(tails) >= self.max_active:
                    break
                if in_use + j.footprint <= self.budget:
                    waiting.remove(j)
                    settle()
                    self.batch.add(j.chain)
                    j.admitted = now
                    in_use += j.footprint
                    active.append(j)
                elif now - j.built >= self.overtake_s:
                    blocked = True                     # nothing younger goes first
                if blocked:
                    break
            if not active:
                if not tails:
                    time.sleep(0.0005)
                else:
                    time.sleep(0.0002)
                continue
            peak_active = max(peak_active, len(active) + len(tails))
            peak_in_use = max(peak_in_use, in_use)
            # jobs with less than a block left leave the batch and finish on
            # their own chains (side stream), after the batch's queued work
            short = [j for j in active if j.remaining < self.block]
            if short:
                settle()
                for j in short:
                    active.remove(j)
                    self.batch.remove(j.chain)
                    j.chain.run(j.remaining, stream=self.side)
                    ev = torch.cuda.Event()
                    ev.record(self.side)
                    j.tail = ev
                    attempts += j.remaining * j.sites
                    j.remaining = 0
                    tails.append(j)
                if not active:
                    continue
            ts = time.perf_counter()
            self.batch.run(self.block, stream=self.stream)
            ticks += 1
            attempts += self.block * sum(j.sites for j in active)
            for j in active:
                j.remaining -= self.block
            # wait for the GPU only if the next tick changes the membership
            # (a job runs out, or one can be admitted); otherwise enqueue on
            inflight = True
            if any(j.remaining < self.block for j in active) or (waiting and in_use + min(
                    w.footprint for w in waiting) <= self.budget) or self._cancel or not built.empty():
                settle()
            busy += time.perf_counter() - ts
        self.stream.synchronize()
        self.side.synchronize()
        wall = time.perf_counter() - t0
        for th in threads:
            th.join()
        ok = [j for j in finished if j.status == "ok"]
        lat = np.array([j.done - j.req.arrival for j in ok]) if ok else np.zeros(1)
        stats = {"requests": n, "completed": len(ok), "cancelled": sum(j.status == "cancelled" for j in finished),
                 "failed": sum(j.status.startswith("failed") for j in finished), "wall_s": wall,
                 "gpu_busy_s": busy, "ticks": ticks, "attempts": attempts,
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
