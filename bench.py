#!/usr/bin/env python
"""Throughput benchmark of the colour-class heat-bath sampler.

Default workload: uniform domino tilings of the Aztec diamond of order 2048
(8,384,513 flip attempts per sweep), all-horizontal start, seed 7, 10^5
heat-bath sweeps per step with edge-density samples every 100 sweeps after a
5 x 10^4 burn-in, then the height function, the north/south/east/west
densities and the state hash.  Other single-chain workloads (--workload):
aztec32 (order 32, 10^4 sweeps, seed 1), hexagon1024 (lozenge tilings of the
1024 x 1024 x 1024 hexagon at q = 0.9995, 5 x 10^4 sweeps, seed 11) and
dwbc2048 (six-vertex N = 2048 with domain-wall boundary at a = b = 1,
c = sqrt 2, 5 x 10^4 sweeps, seed 11); plus batch (4096 chains) and serve
(Poisson request stream).

Metric: flip attempts per second (whole job, all ranks), with the dominant
kernel's achieved fraction of the HBM roofline.  One process per GPU; for
N > 1 (torchrun) every rank runs an independent replica of the workload
(weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload aztec2048|aztec32|hexagon1024|dwbc2048|batch|serve]

--impl reference times the CPU oracle (the plain single-threaded reference
sampler) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flip attempts/s"
SQRT2 = 2.0 ** 0.5


# Single-chain workloads: domain, weights, seed and sweeps per step.
# `oracle_sweeps` bounds the CPU oracle's sample per reference-arm step and
# `baseline_sweeps` the cpu_baseline sample (about 10-30 s of CPU work).
WORKLOADS = {
    "aztec2048": dict(name="aztec_diamond_n2048_uniform_domino", kind="aztec", size=(2048,), seed=7,
                      sweeps=100_000, density=(100, 50_000), oracle_sweeps=16, baseline_sweeps=100),
    "aztec32": dict(name="aztec_diamond_n32_uniform_domino", kind="aztec", size=(32,), seed=1,
                    sweeps=10_000, density=None, oracle_sweeps=10_000, baseline_sweeps=10_000),
    "hexagon1024": dict(name="hexagon_1024x1024x1024_q0.9995_lozenge", kind="hexagon", size=(1024, 1024, 1024),
                        seed=11, sweeps=50_000, q=0.9995, density=None, oracle_sweeps=32, baseline_sweeps=100),
    "dwbc2048": dict(name="sixvertex_dwbc_n2048_a1_b1_c_sqrt2", kind="dwbc", size=(2048,), seed=11,
                     sweeps=50_000, w6=(1.0, 1.0, 1.0, 1.0, SQRT2, SQRT2), density=None,
                     oracle_sweeps=16, baseline_sweeps=60),
}
UNIFORM_T = 1 << 31
KERNEL_SOURCES = ["paper_1804_07250_gb300/csrc/tl_resident.cu", "paper_1804_07250_gb300/csrc/tl_device.cuh"]
REG_SOURCES = ["paper_1804_07250_gb300/csrc/tl_regdom.cu", "paper_1804_07250_gb300/csrc/tl_device.cuh"]
# plan kernel -> (ncu kernel name, sources whose hash keys the recorded traffic)
RESIDENT_KERNELS = {2: ("resident_kernel", KERNEL_SOURCES), 3: ("regdom_kernel", REG_SOURCES)}
BATCH_SOURCES = ["paper_1804_07250_gb300/csrc/tl_batch.cu", "paper_1804_07250_gb300/csrc/tl_device.cuh"]


def kernel_hash(sources=None):
    import hashlib
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, sources=None, plan=None):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources (and the recorded plan fields, if any) still match the ones it
    was captured with."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(workload)
    except Exception:
        return None
    if not rec or rec.get("kernel_hash") != kernel_hash(sources):
        return None
    for k, v in rec.get("plan", {}).items():
        if plan is None or plan.get(k) != v:
            return None
    return rec.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_setup(wl):
    """Starting state and threshold keywords of a workload, from the oracle."""
    import oracle as O
    if wl["kind"] == "aztec":
        return O.DOMINO, O.aztec(*wl["size"]), {"t_scalar": UNIFORM_T}
    if wl["kind"] == "hexagon":
        t_add, _ = O.lozenge_thresholds(wl["q"])
        return O.LOZENGE, O.hexagon(*wl["size"]), {"t_scalar": t_add}
    return O.SIXV, O.dwbc(*wl["size"]), {"t16": O.sixv_thresholds(wl["w6"])}


def oracle_rate(wl, sweeps: int, sites: int, state=None):
    """Attempts/s of the oracle over `sweeps` sweeps; continues from `state`
    (lattice, array, sweep0) when given so that repeated samples do not all
    time the first sweeps after the start."""
    import oracle as O
    if state is None:
        lat, st, kw = oracle_setup(wl)
        state = [lat, st, kw, 0]
    lat, st, kw, s0 = state
    t0 = time.perf_counter()
    O.sweeps(lat, st, seed=wl["seed"], stream=0, sweep0=s0, k=sweeps, **kw)
    dt = time.perf_counter() - t0
    state[3] = s0 + sweeps
    return sites * sweeps / dt, dt, state


def workload_sites(wl):
    """Interior sites: Aztec n^2 + (n-1)^2, six-vertex (N-1)^2, hexagon
    ab + bc + ca - a - b - c + 1."""
    if wl["kind"] == "aztec":
        n = wl["size"][0]
        return n * n + (n - 1) ** 2
    if wl["kind"] == "dwbc":
        return (wl["size"][0] - 1) ** 2
    a, b, c = wl["size"]
    return a * b + b * c + c * a - a - b - c + 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    wl = WORKLOADS[args.workload]
    sites = workload_sites(wl)
    k = wl["oracle_sweeps"]
    state = None
    for _ in range(args.warmup):
        _, _, state = oracle_rate(wl, 1, sites, state)
    total = 0.0
    for _ in range(args.steps):
        _, dt, state = oracle_rate(wl, k, sites, state)
        total += dt
    value = args.steps * k * sites / total
    sample = "%d sweeps per step of the %s workload (of %d)" % (k, wl["name"], wl["sweeps"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["name"], "size": list(wl["size"]), "sweeps_per_step": k,
                       "seed": wl["seed"]},
            "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_1804_07250_gb300 as T

    wl = WORKLOADS[args.workload]
    SWEEPS = args.sweeps or wl["sweeps"]
    ctx = T.Context(local)
    if wl["kind"] == "aztec":
        dom = T.Domain.aztec(*wl["size"])
        th = T.thresholds(scalar=UNIFORM_T)
        thr_desc = UNIFORM_T
    elif wl["kind"] == "hexagon":
        dom = T.Domain.hexagon(*wl["size"])
        t_add, _ = T.lozenge_thresholds(wl["q"])
        th = T.thresholds(scalar=t_add)
        thr_desc = {"q": wl["q"], "t_add": t_add}
    else:
        dom = T.Domain.dwbc(*wl["size"])
        t16 = T.sixv_thresholds(wl["w6"])
        th = T.thresholds(table16=t16)
        thr_desc = {"w6": list(wl["w6"]), "t16": [int(v) for v in t16]}
    info = dom.info
    stream = torch.cuda.Stream()
    from paper_1804_07250_gb300 import replicas
    # every rank samples its own replica: same workload, its own stream id
    chain = T.Chain(ctx, dom, seed=wl["seed"], stream_id=replicas.replica_stream_id(0, rank, world), th=th)
    if args.kernel or args.spl or args.halo or args.threads or args.npre:
        chain.set_plan(args.kernel, args.spl, args.halo, args.threads, args.npre)
    hshape = dom.height_shape
    density = wl["density"]
    height_dev = torch.empty(hshape, dtype=torch.int32, device="cuda")
    nsew_dev = (torch.empty((4, info.height - 1, info.width - 1), dtype=torch.float64, device="cuda")
                if density else None)
    hash_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step(s, ev=None):
        chain.reset(stream=s)
        if density:
            chain.density_begin(*density)
        if ev:
            ev[0].record(s)
        chain.run(SWEEPS, stream=s)
        if ev:
            ev[1].record(s)
        chain.read_height(height_dev, stream=s)
        if density:
            chain.read_nsew(nsew_dev, stream=s)
        chain.state_hash(out=hash_dev, stream=s)

    for _ in range(args.warmup):
        step(stream)
    stream.synchronize()
    chain.sync(stream)
    ref_hash = int(hash_dev.cpu().numpy().view(np.uint64)[0])

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = chain.launches
    total_ms, run_ms, run_launches = 0.0, 0.0, 0
    for _ in range(args.steps):
        flush.zero_()                      # L2 flush between timed steps (not timed)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(stream, (r0, r1))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        total_ms += e0.elapsed_time(e1)
        run_ms += r0.elapsed_time(r1)
        run_launches += 1
    clocks = sampler.stop()
    chain.sync(stream)
    launches = chain.launches - launches0
    got_hash = int(hash_dev.cpu().numpy().view(np.uint64)[0])
    assert got_hash == ref_hash, "steps are not deterministic"
    total_ms = replicas.max_over_ranks(total_ms, dist, device="cuda")   # the slowest rank's time
    attempts_step = info.sites * SWEEPS
    value = world * attempts_step * args.steps / (total_ms / 1e3)

    # dominant kernel: the sweep launches of each step, timed with CUDA
    # events on their stream
    plan = chain.plan()
    if plan["kernel"] in RESIDENT_KERNELS:
        # the library splits a run into launches of at most spl sweeps and at
        # most 60000 * halo / passes sweeps (16-bit exchange tags)
        per = max(1, 60000 * plan["halo"] // info.passes)
        if plan["sweeps_per_launch"]:
            per = min(per, plan["sweeps_per_launch"])
        k_launches_per_run = -(-SWEEPS // per)
    else:
        k_launches_per_run = SWEEPS * info.passes
    k_ms = run_ms / run_launches / k_launches_per_run
    bytes_per_sweep = 2 * info.edges / 8
    alg_bytes_launch = bytes_per_sweep * SWEEPS / k_launches_per_run
    peak, peak_kind = peaks()
    achieved = alg_bytes_launch / (k_ms / 1e3) / 1e9
    kname, ksrc = RESIDENT_KERNELS.get(plan["kernel"], ("pass_global_kernel", KERNEL_SOURCES))
    # the recorded traffic is of the workload's own launches: none for
    # another sweep count or plan
    traffic = recorded_traffic(wl["name"], ksrc, {"kernel": plan["kernel"]}) \
        if plan["kernel"] in RESIDENT_KERNELS and SWEEPS == wl["sweeps"] else None

    # end to end through the C-ABI: every step copies its start state in from
    # page-locked host memory and its results (state, heights and, with
    # densities, the N/S/E/W densities) out to page-locked host memory.  The
    # library writes the results into device buffers on the compute stream;
    # their copies to the host run on a copy stream, overlapping the next
    # step's sweeps, with the buffers alternating by step parity.  The timed
    # region ends when the last step's copies have landed.
    def pinned(shape, dtype):
        return torch.empty(tuple(shape), dtype=dtype, pin_memory=True)

    nshape = (4, info.height - 1, info.width - 1)
    init_host = pinned(dom.canon_shape, torch.uint8)
    init_host.numpy()[...] = dom.initial_state()
    init_dev = torch.empty(dom.canon_shape, dtype=torch.uint8, device="cuda")
    res_dev = [(torch.empty(dom.canon_shape, dtype=torch.uint8, device="cuda"),
                torch.empty(hshape, dtype=torch.int32, device="cuda"),
                torch.empty(nshape, dtype=torch.float64, device="cuda") if density else None) for _ in range(2)]
    res_host = [(pinned(dom.canon_shape, torch.uint8), pinned(hshape, torch.int32),
                 pinned(nshape, torch.float64) if density else None) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [None, None]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        b = i & 1
        with torch.cuda.stream(stream):
            init_dev.copy_(init_host, non_blocking=True)  # host -> device
        chain.reset(stream=stream)
        chain.write_state(init_dev, stream=stream)        # validated on the device
        if density:
            chain.density_begin(*density)
        chain.run(SWEEPS, stream=stream)
        if copied[b] is not None:
            stream.wait_event(copied[b])                  # step i - 2's copies have left buffer b
        s_dev, h_dev, n_dev = res_dev[b]
        chain.read_state(s_dev, stream=stream)
        chain.read_height(h_dev, stream=stream)
        if density:
            chain.read_nsew(n_dev, stream=stream)
        ready = torch.cuda.Event()
        ready.record(stream)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):              # device -> host
            for src, dst in zip(res_dev[b], res_host[b]):
                if src is not None:
                    dst.copy_(src, non_blocking=True)
        copied[b] = torch.cuda.Event()
        copied[b].record(copy_stream)
    torch.cuda.synchronize()
    chain.sync(stream)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * attempts_step * e2e_steps / e2e_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        k = wl["baseline_sweeps"]
        r, dt, _ = oracle_rate(wl, k, info.sites)
        cpu = {"value": r, "unit": "attempts/s", "cores": 1, "kind": "oracle",
               "sample": "%d sweeps of the %s workload from its start state (%.1f s)" % (k, wl["name"], dt)}

    if rank == 0:
        cfg = {"workload": wl["name"], "size": list(wl["size"]), "sites": info.sites,
               "sweeps_per_step": SWEEPS, "threshold": thr_desc, "seed": wl["seed"],
               "l2": "flushed between steps (256 MB write); state is L2-sized",
               "parallelism": "replicas" if world > 1 else "single"}
        if density:
            cfg.update(density_stride=density[0], burn_in=density[1])
        d2h = int(sum(t.numel() * t.element_size() for t in res_host[0] if t is not None))
        line = {"metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic", "config": cfg,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                             "traffic": traffic, "kernel": kname, "kernel_ms": k_ms,
                             "alg_bytes_per_launch": alg_bytes_launch,
                             "us_per_sweep": 1e3 * run_ms / run_launches / SWEEPS,
                             "kernel_hash": kernel_hash(ksrc), "plan": plan},
                "clocks": clocks,
                "gpu_launches": launches,
                "e2e": {"value": e2e_value, "unit": "attempts/s",
                        "h2d_bytes_per_step": int(init_host.numel() * init_host.element_size()),
                        "d2h_bytes_per_step": d2h},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Batched workload: 4096 Aztec chains, orders U{16..512} (seed 3), per-site
# heat-bath thresholds from log-normal (sigma 0.5) dual-edge weights, 10^4
# sweeps per step in CUDA-graph blocks of 100; compared with one launch per
# chain per R sweeps on the same GPU.
# ---------------------------------------------------------------------------
BATCH_CHAINS, BATCH_SWEEPS, BATCH_BLOCK = 4096, 10_000, 100


def build_batch(T, ctx, nchains):
    import numpy as np
    orders = np.random.default_rng(3).integers(16, 513, size=nchains)
    chains, sites, edges = [], 0, 0
    for i, n in enumerate(orders):
        dom = T.Domain.aztec(int(n))
        W = 2 * int(n) + 1
        z = np.random.default_rng([3, i]).standard_normal((2, W, W))
        t = dom.domino_thresholds(np.exp(0.5 * z))
        chains.append(T.Chain(ctx, dom, seed=3, stream_id=i, th=T.thresholds(site=t)))
        sites += dom.info.sites
        edges += dom.info.edges
    return chains, orders, sites, edges


def run_batch(args):
    import numpy as np
    import torch
    import paper_1804_07250_gb300 as T
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = T.Context(local)
    t0 = time.perf_counter()
    chains, orders, sites, edges = build_batch(T, ctx, args.chains)
    setup_s = time.perf_counter() - t0
    b = T.Batch(ctx, chains)
    stream = torch.cuda.Stream()
    plan = b.autotune(trial_sweeps=48, stream=stream)
    b.set_plan(graph_block=BATCH_BLOCK)
    for _ in range(args.warmup):
        b.run(BATCH_BLOCK, stream=stream)
    stream.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = b.launches
    total_ms, step_ms = 0.0, []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(args.batch_sweeps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    total_ms = sum(step_ms)
    clocks = sampler.stop()
    launches = b.launches - l0
    value = sites * args.batch_sweeps * args.steps / (total_ms / 1e3)
    # one launch per chain per R sweeps, same kernel
    kpc = 2 * plan["sweeps_per_launch"] * 5
    per_chain = None
    if not args.no_per_chain:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run_per_chain(kpc, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        per_chain = sites * kpc / (e0.elapsed_time(e1) / 1e3)
    # 32 sampled chains (all of them if fewer) against the same chain run
    # alone for the same number of sweeps: the batch must not change results
    stream.synchronize()
    hb = b.hashes()
    pick = np.sort(np.random.default_rng(11).choice(len(chains), size=min(32, len(chains)), replace=False))
    same = 0
    for i in pick:
        c = chains[int(i)]
        alone = T.Chain(ctx, c.domain, seed=3, stream_id=int(i), th=T.thresholds(site=c.domain.domino_thresholds(
            np.exp(0.5 * np.random.default_rng([3, int(i)]).standard_normal(
                (2, 2 * int(orders[i]) + 1, 2 * int(orders[i]) + 1))))))
        alone.run(c.sweep)
        same += int(alone.state_hash() == int(hb[int(i)]))
        alone.close()
    assert same == len(pick), "batched chains differ from the same chains run alone"
    peak, peak_kind = peaks()
    us_sweep = 1e3 * total_ms / (args.steps * args.batch_sweeps)
    state_bytes = 2 * edges / 8
    packed_mb = sum(c.domain.info.packed_bytes for c in chains) / 1e6
    thr_mb = 4 * sites / 1e6
    workload = "batched_%d_aztec_chains_n16_512_lognormal" % args.chains
    bplan = b.plan()
    traffic = recorded_traffic(workload, BATCH_SOURCES, bplan)
    line = {"metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload,
                       "chains": args.chains, "sites_per_sweep": int(sites),
                       "mean_n2": float(np.mean(orders.astype(np.float64) ** 2)),
                       "sweeps_per_step": args.batch_sweeps, "graph_block": BATCH_BLOCK,
                       "plan": bplan, "autotuned": plan, "setup_s": setup_s,
                       "l2": "state (%.0f MB) and thresholds (%.0f MB) %s than L2 (129 MB); no flush" %
                             (packed_mb, thr_mb, "larger" if packed_mb + thr_mb > 129 else "smaller")},
            "roofline": {"bound": "hbm", "achieved": state_bytes / (us_sweep * 1e-6) / 1e9, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": state_bytes / (us_sweep * 1e-6) / 1e9 / peak,
                         "us_per_sweep": us_sweep, "traffic": traffic, "kernel": "batch_kernel",
                         "sweeps_per_launch": bplan["sweeps_per_launch"],
                         "alg_bytes_per_launch": state_bytes * bplan["sweeps_per_launch"]},
            "batched_vs_per_chain": None if per_chain is None else
                {"batched": value, "per_chain": per_chain, "speedup": value / per_chain, "per_chain_sweeps": kpc},
            "sampled_check": {"chains": int(len(pick)), "equal_to_alone": same,
                              "sweeps_each": int(chains[int(pick[0])].sweep)},
            "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Served workload: Poisson arrivals (mean 200 requests/s, seed 5) of sampling
# jobs (a third each Aztec n in [32, 2048], hexagons with sides in [16, 512],
# six-vertex domain wall N in [32, 1024]; uniform or log-normal weights;
# 10^3..10^5 sweeps log-uniform), admitted against an 80 GB budget.
# ---------------------------------------------------------------------------
def run_serve(args):
    import numpy as np
    import torch
    import paper_1804_07250_gb300 as T
    from paper_1804_07250_gb300 import serve
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = T.Context(local)
    out = {}
    for label, rate in (("rate", args.rate), ("half_rate", args.rate / 2)):
        reqs = serve.make_requests(args.requests, rate=rate, seed=5)
        srv = serve.Server(ctx, budget_bytes=int(args.budget_gb * 1e9))
        sampler = ClockSampler(local)
        sampler.start()
        done, stats = srv.run(reqs, keep_chains=False)
        stats["clocks"] = sampler.stop()
        stats["offered_attempts_per_s"] = float(sum(
            r.sweeps * (T.Domain.aztec(*r.size).info.sites if r.kind == "aztec" else
                        T.Domain.hexagon(*r.size).info.sites if r.kind == "hexagon" else
                        (r.size[0] - 1) ** 2) for r in reqs) / reqs[-1].arrival)
        out[label] = {"rate_per_s": rate, **stats}
        if label == "rate":
            rng = np.random.default_rng(11)
            pick = rng.choice(len(done), size=min(args.check, len(done)), replace=False)
            same = sum(int(done[i].status == "ok" and done[i].result_hash == serve.alone_hash(ctx, done[i].req))
                       for i in pick)
            out["alone_vs_mixed"] = {"checked": int(len(pick)), "identical": int(same)}
    main_stats = out["rate"]
    line = {"metric": METRIC, "value": main_stats["attempts_per_s"], "unit": "attempts/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * main_stats["wall_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "served_poisson_%g_per_s_%d_requests" % (args.rate, args.requests),
                       "budget_gb": args.budget_gb, "block": 100},
            "clocks": main_stats.get("clocks"),
            "serve": out}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Exact samplers: domino shuffling of the Aztec diamond of order 2048, and
# coupling from the past on the Aztec diamond of order 128 (uniform).
# ---------------------------------------------------------------------------
EXACT = {"shuffle2048": ("aztec_diamond_n2048_domino_shuffling", 2048),
         "shuffle512": ("aztec_diamond_n512_domino_shuffling", 512),
         "cftp_aztec128": ("aztec_diamond_n128_coupling_from_the_past", 128)}


def run_exact(args):
    import numpy as np
    import torch
    import paper_1804_07250_gb300 as T
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = T.Context(local)
    name, n = EXACT[args.workload]
    stream = torch.cuda.Stream()
    shuffle = args.workload.startswith("shuffle")
    dom = None if shuffle else T.Domain.aztec(n)
    th = T.thresholds(scalar=UNIFORM_T)
    out_dev = torch.empty((2, 2 * n + 1, 2 * n + 1), dtype=torch.uint8, device="cuda")

    def one(seed):
        if shuffle:
            T.aztec_shuffle(ctx, n, seed=seed, stream_id=rank, out=out_dev, stream=stream)
            return 0
        _, t_used = T.cftp(ctx, dom, seed=seed, stream_id=rank, th=th, t0=64, out=out_dev, stream=stream)
        return t_used

    for w in range(args.warmup):
        one(10_000 + w)
    sampler = ClockSampler(local)
    sampler.start()
    t0 = time.perf_counter()
    used = [one(s) for s in range(args.steps)]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    clocks = sampler.stop()
    value = world * args.steps / dt
    # work: shuffling touches sum_k (2k)^2 cells; CFTP runs 2 chains over
    # 64 + 128 + ... + T sweeps of n^2 + (n-1)^2 sites
    sites = n * n + (n - 1) ** 2
    if shuffle:
        cells = sum((2 * k) ** 2 for k in range(1, n + 1))
        extra = {"cell_updates_per_s": cells * args.steps / dt}
    else:
        sweeps = [2 * (2 * t - 64) for t in used]
        extra = {"flip_attempts_per_s": sites * sum(sweeps) / dt, "T_used": used}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        if shuffle:
            m = 96
            t1 = time.perf_counter()
            O.aztec_shuffle(m, 1)
            d1 = time.perf_counter() - t1
            cells_m = sum((2 * k) ** 2 for k in range(1, m + 1))
            cpu = {"value": cells_m / d1, "unit": "cell updates/s", "cores": 1, "kind": "oracle",
                   "sample": "one oracle shuffle of order %d (%.1f s)" % (m, d1)}
        else:
            r, d1, _ = oracle_rate(WORKLOADS["aztec2048"] | {"size": (n,)}, 400, sites)
            cpu = {"value": r, "unit": "flip attempts/s", "cores": 1, "kind": "oracle",
                   "sample": "400 oracle sweeps of the order-%d diamond (%.1f s)" % (n, d1)}
    if rank == 0:
        line = {"metric": "exact samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "config": {"workload": name, "n": n, "seeds": "0..steps-1",
                                                "l2": "state fits in L2; no flush (each step allocates its buffers)"},
                **extra, "clocks": clocks, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)


def free_port() -> int:
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(nprocs: int) -> int:
    """Re-run this command as `nprocs` ranks (one process per GPU) under
    torch.distributed.run on 127.0.0.1, when it was started as a single
    process with --gpus N > 1; returns the launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=%d" % nprocs,
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.abspath(__file__),
           *sys.argv[1:]]
    return subprocess.call(cmd)


def run_dry(args):
    """Launcher check without GPUs: every rank times a small oracle replica
    (its own stream id), the slowest rank's time is taken, and rank 0 prints
    one line.  gloo on CPU, NCCL when every rank has a GPU."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    use_cuda = torch.cuda.is_available()
    if world > 1:
        if use_cuda:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if use_cuda else "gloo")
    import oracle as O
    from paper_1804_07250_gb300 import replicas
    t0 = time.perf_counter()
    st = O.aztec(16)
    O.sweeps(O.DOMINO, st, seed=7, stream=replicas.replica_stream_id(0, rank, world), k=20, t_scalar=UNIFORM_T)
    dt = replicas.max_over_ranks(time.perf_counter() - t0, dist if world > 1 else None,
                                 device="cuda" if use_cuda else "cpu")
    hashes = replicas.gather_results(O.state_hash(st), dist if world > 1 else None)
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "ranks_seen": len(hashes),
                          "distinct_streams": len(set(hashes)), "slowest_rank_s": dt}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 per-pass, 2 resident")
    ap.add_argument("--spl", type=int, default=0, help="sweeps per launch (0 auto)")
    ap.add_argument("--halo", type=int, default=0, help="resident kernel halo (0 auto)")
    ap.add_argument("--threads", type=int, default=0, help="resident kernel threads (0 auto)")
    ap.add_argument("--npre", type=int, default=0, help="random planes generated ahead (0 auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="sweeps per step instead of the workload's (short runs for profiling only)")
    ap.add_argument("--workload", choices=[*WORKLOADS, *EXACT, "batch", "serve"], default="aztec2048")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=80.0)
    ap.add_argument("--check", type=int, default=50)
    ap.add_argument("--chains", type=int, default=BATCH_CHAINS)
    ap.add_argument("--batch-sweeps", type=int, default=BATCH_SWEEPS)
    ap.add_argument("--no-per-chain", action="store_true",
                    help="batch: skip the one-launch-per-chain comparison")
    ap.add_argument("--dry-run", action="store_true",
                    help="check the rank launcher only (no GPU needed): a small oracle replica per rank")
    args = ap.parse_args()
    # --gpus N started as one process: become N ranks (the driver may also
    # start the ranks itself under torchrun, with WORLD_SIZE set)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus))
    if args.dry_run:
        run_dry(args)
        return
    if args.workload == "batch" and args.impl == "ours":
        run_batch(args)
        return
    if args.workload == "serve" and args.impl == "ours":
        run_serve(args)
        return
    if args.workload in EXACT and args.impl == "ours":
        run_exact(args)
        return
    if args.impl == "reference":
        if args.workload not in WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single-chain workloads"}))
            return
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
