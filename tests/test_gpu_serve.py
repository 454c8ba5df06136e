"""Serving: requests admitted into a running batch (continuous batching) must
give exactly the result they give alone, and the loop must report latencies."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_07250_gb300 as T
    from paper_1804_07250_gb300 import serve
    return T, serve


def test_served_results_equal_alone(S):
    T, serve = S
    ctx = T.Context(0)
    reqs = serve.make_requests(40, rate=400.0, seed=5, aztec=(16, 90), hexagon=(6, 40), dwbc=(12, 70),
                               sweeps=(30, 400))
    srv = serve.Server(ctx, budget_bytes=2 << 30, block=50, tile_rows=32, sweeps_per_launch=3)
    done, stats = srv.run(reqs)
    assert len(done) == len(reqs) and stats["peak_active"] > 1
    assert 0 < stats["p50_latency_s"] <= stats["p99_latency_s"]
    by_id = {j.req.rid: j for j in done}
    for r in reqs:
        assert by_id[r.rid].result_hash == serve.alone_hash(ctx, r), "request %d" % r.rid


def test_admission_respects_budget(S):
    T, serve = S
    ctx = T.Context(0)
    reqs = serve.make_requests(12, rate=1000.0, seed=9, aztec=(40, 60), hexagon=(20, 30), dwbc=(30, 40),
                               sweeps=(100, 200))
    one = max(serve.footprint(T.Domain.aztec(60), True), serve.footprint(T.Domain.hexagon(30, 30, 30), True),
              serve.footprint(T.Domain.dwbc(40), False))
    srv = serve.Server(ctx, budget_bytes=2 * one, block=50, tile_rows=32, sweeps_per_launch=2)
    done, stats = srv.run(reqs)
    assert len(done) == len(reqs)
    assert 0 < stats["peak_in_use_bytes"] <= 2 * one
    assert stats["peak_active"] < len(reqs)      # the budget made later requests wait


def test_lognormal_device_thresholds(S):
    import torch
    T, serve = S
    d = T.Domain.aztec(50)
    t = torch.empty((d.info.height, d.info.width), dtype=torch.int32, device="cuda")
    d.lognormal_thresholds_device(0.0, 7, t)          # sigma 0: every weight is 1
    assert bool((t.cpu().numpy().view(np.uint32) == 1 << 31).all())
    d.lognormal_thresholds_device(0.5, 7, t)
    a = t.cpu().numpy().view(np.uint32).astype(np.float64) / 2 ** 32
    d.lognormal_thresholds_device(0.5, 7, t)
    assert np.array_equal(a, t.cpu().numpy().view(np.uint32).astype(np.float64) / 2 ** 32)  # deterministic
    inner = a[2:-2, 2:-2]
    assert 0.45 < inner.mean() < 0.55 and inner.std() > 0.1


def test_faults_cancel_and_failed_build_leave_others_unchanged(S):
    # host-side faults: a request cancelled while it runs, one cancelled
    # before it is admitted, and two whose build fails (as an allocation
    # failure would); every other request still equals its result alone
    T, serve = S
    ctx = T.Context(0)
    reqs = serve.make_requests(24, rate=300.0, seed=13, aztec=(16, 80), hexagon=(6, 30), dwbc=(12, 60),
                               sweeps=(200, 2000))
    bad = {reqs[3].rid, reqs[10].rid}

    def fault(r):
        return T.TilingError(T.TL_ENOMEM, "injected allocation failure") if r.rid in bad else None

    srv = serve.Server(ctx, budget_bytes=2 << 30, block=50, tile_rows=32, sweeps_per_launch=2, build_fault=fault)
    srv.cancel(reqs[20].rid)                 # before it arrives
    import threading
    late = reqs[5].rid
    threading.Timer(0.05, srv.cancel, args=(late,)).start()   # most likely while it runs
    done, stats = srv.run(reqs)
    by_id = {j.req.rid: j for j in done}
    assert len(done) == len(reqs)
    assert by_id[reqs[20].rid].status == "cancelled"
    assert by_id[late].status in ("cancelled", "ok")
    for rid in bad:
        assert by_id[rid].status.startswith("failed") and "injected" in by_id[rid].status
    assert stats["failed"] == 2 and stats["completed"] + stats["cancelled"] + stats["failed"] == len(reqs)
    for r in reqs:
        j = by_id[r.rid]
        if j.status == "ok":
            assert j.result_hash == serve.alone_hash(ctx, r), "request %d" % r.rid


def test_overtaking_admits_small_jobs_past_a_large_one(S):
    # small jobs hold most of the budget when a large one arrives: later
    # small jobs that fit are admitted before it (budget-aware overtaking),
    # until it has waited overtake_s; then it goes first, and completes
    T, serve = S
    ctx = T.Context(0)
    small = [serve.Request(rid=i, arrival=0.0005 * i, kind="aztec", size=(24,), weights="uniform", sweeps=3000,
                           seed=21) for i in range(12)]
    big = serve.Request(rid=99, arrival=0.0016, kind="aztec", size=(150,), weights="uniform", sweeps=300, seed=21)
    fs = serve.footprint(T.Domain.aztec(24), False)
    fb = serve.footprint(T.Domain.aztec(150), False)
    budget = fb + fs                     # the big job needs the small ones all but gone
    srv = serve.Server(ctx, budget_bytes=budget, block=50, tile_rows=32, sweeps_per_launch=2,
                       overtake_s=0.2, workers=1)
    done, stats = srv.run(small[:4] + [big] + small[4:])
    assert stats["completed"] == 13
    by_id = {j.req.rid: j for j in done}
    assert any(j.req.arrival > big.arrival and j.admitted < by_id[99].admitted for j in done if j.req.rid != 99)
    assert by_id[99].result_hash == serve.alone_hash(ctx, big)
    for r in small:
        assert by_id[r.rid].result_hash == serve.alone_hash(ctx, r)

