"""Batched chains: every chain of a batch must end bit-identical to the same
chain run on its own and to the CPU oracle, whatever the plan (tile height,
sweeps per launch, graph blocks) and whether launched batched or one launch
per chain."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
SQ2 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_07250_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctx(T):
    return T.Context(0)


def _specs():
    rng = np.random.default_rng(3)
    out = []
    for i, n in enumerate([5, 17, 40, 77, 130]):
        W = 2 * n + 1
        w = np.exp(0.5 * rng.standard_normal((2, W, W)))
        out.append(("aztec", (n,), dict(site=O.domino_thresholds(w))))
    out.append(("aztec", (64,), dict(scalar=1 << 31)))
    out.append(("rect", (90, 33), dict(scalar=1 << 31)))
    out.append(("hex", (20, 30, 25), dict(scalar=O.lozenge_thresholds(0.9995)[0])))
    out.append(("hex", (7, 5, 9), dict(scalar=O.lozenge_thresholds(1.3)[0])))
    out.append(("dwbc", (50,), dict(t16=O.sixv_thresholds(SQ2))))
    out.append(("dwbc", (9,), dict(t16=O.sixv_thresholds([0.7, 1.3, 0.4, 1.9, 1.1, 0.6]))))
    return out


def _make(T, ctx, spec, stream_id):
    kind, args, th = spec
    dom = {"aztec": T.Domain.aztec, "rect": T.Domain.rect, "hex": T.Domain.hexagon,
           "dwbc": T.Domain.dwbc}[kind](*args)
    if "t16" in th:
        t = T.thresholds(table16=th["t16"])
    elif "site" in th:
        t = T.thresholds(site=th["site"])
    else:
        t = T.thresholds(scalar=th["scalar"])
    return T.Chain(ctx, dom, seed=2024, stream_id=stream_id, th=t)


def _oracle(spec, stream_id, k):
    kind, args, th = spec
    st = {"aztec": O.aztec, "rect": O.rect, "hex": O.hexagon, "dwbc": O.dwbc}[kind](*args)
    lat = {"aztec": O.DOMINO, "rect": O.DOMINO, "hex": O.LOZENGE, "dwbc": O.SIXV}[kind]
    kw = {"t16": th["t16"]} if "t16" in th else ({"t_site": th["site"]} if "site" in th else {"t_scalar": th["scalar"]})
    O.sweeps(lat, st, seed=2024, stream=stream_id, k=k, **kw)
    return st


@pytest.mark.parametrize("tile_rows,R,block,per_chain,threads", [
    (64, 2, 100, False, 256), (8, 1, 100, False, 256), (16, 3, 6, False, 256), (32, 4, 8, False, 256),
    (5, 2, 100, True, 256), (64, 2, 100, False, 128), (16, 3, 6, False, 128), (5, 2, 100, True, 128)])
def test_batch_matches_alone_and_oracle(T, ctx, tile_rows, R, block, per_chain, threads):
    import torch
    specs = _specs()
    chains = [_make(T, ctx, sp, 100 + i) for i, sp in enumerate(specs)]
    b = T.Batch(ctx, chains)
    b.set_plan(tile_rows, R, block, threads)
    assert b.plan()["threads"] == threads
    stream = torch.cuda.Stream()
    k1, k2 = 13, 24
    (b.run_per_chain if per_chain else b.run)(k1, stream=stream)
    (b.run_per_chain if per_chain else b.run)(k2, stream=stream)
    stream.synchronize()
    hb = b.hashes()
    for i, (sp, ch) in enumerate(zip(specs, chains)):
        assert ch.sweep == k1 + k2
        alone = _make(T, ctx, sp, 100 + i)
        alone.run(k1 + k2)
        assert int(hb[i]) == alone.state_hash(), "chain %d differs from running alone" % i
        st = _oracle(sp, 100 + i, k1 + k2)
        assert np.array_equal(ch.read_state(), st), "chain %d differs from the oracle" % i


def test_batch_autotune_keeps_results(T, ctx):
    import torch
    specs = _specs()
    chains = [_make(T, ctx, sp, 300 + i) for i, sp in enumerate(specs)]
    ref = [_make(T, ctx, sp, 300 + i) for i, sp in enumerate(specs)]
    b = T.Batch(ctx, chains)
    stream = torch.cuda.Stream()
    plan = b.autotune(trial_sweeps=4, stream=stream)
    assert plan["tile_rows"] in (32, 64, 128) and plan["sweeps_per_launch"] in (1, 2, 4, 8)
    assert all(c.sweep == 0 for c in chains)
    b.run(20, stream=stream)
    stream.synchronize()
    for c, r in zip(chains, ref):
        r.run(20)
        assert c.state_hash() == r.state_hash()


def test_autotune_cache(T, ctx):
    # a second batch with the same key (lattices, threshold kinds, rows to a
    # power of two, SMs) takes the cached plan without trials
    import time

    import torch
    T.Batch.autotune_cache_clear()
    specs = _specs()
    stream = torch.cuda.Stream()
    b1 = T.Batch(ctx, [_make(T, ctx, sp, 700 + i) for i, sp in enumerate(specs)])
    t0 = time.perf_counter()
    p1 = b1.autotune(trial_sweeps=16, stream=stream)
    first = time.perf_counter() - t0
    chains = [_make(T, ctx, sp, 800 + i) for i, sp in enumerate(specs)]
    b2 = T.Batch(ctx, chains)
    t0 = time.perf_counter()
    p2 = b2.autotune(trial_sweeps=16, stream=stream)
    second = time.perf_counter() - t0
    assert (p2["tile_rows"], p2["sweeps_per_launch"]) == (p1["tile_rows"], p1["sweeps_per_launch"])
    assert second < first / 4
    assert all(c.sweep == 0 for c in chains)
    b2.run(12, stream=stream)
    stream.synchronize()
    for i, (sp, c) in enumerate(zip(specs, chains)):
        assert np.array_equal(c.read_state(), _oracle(sp, 800 + i, 12))
    T.Batch.autotune_cache_clear()
