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
