"""Checkpoint and resume (RandomWalk's state carried across calls, Sec. 2.2).

k + k sweeps in one chain must equal k sweeps, a checkpoint, a restore into
a new context and k more sweeps: same hash, same state, same sweep index,
and both equal to the oracle.  Covers every lattice, per-site thresholds,
the random pass order, and a domain from a boundary path.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from tests.test_gpu_regions_cftp import DOMINO_PATHS

pytestmark = pytest.mark.gpu
SQ2 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_07250_gb300 as T
    return T


def _case(T, name):
    rng = np.random.default_rng(17)
    if name == "aztec_half":
        return T.Domain.aztec(120), O.aztec(120), O.DOMINO, dict(scalar=1 << 31)
    if name == "aztec_site":
        w = np.exp(0.5 * rng.standard_normal((2, 2 * 60 + 1, 2 * 60 + 1)))
        return T.Domain.aztec(60), O.aztec(60), O.DOMINO, dict(site=O.domino_thresholds(w))
    if name == "hexagon":
        return T.Domain.hexagon(40, 30, 50), O.hexagon(40, 30, 50), O.LOZENGE, dict(scalar=O.lozenge_thresholds(0.97)[0])
    if name == "dwbc":
        return T.Domain.dwbc(90), O.dwbc(90), O.SIXV, dict(t16=O.sixv_thresholds(SQ2))
    steps = DOMINO_PATHS["U"]()
    st = O.tiling_by_search(O.DOMINO, O.region_from_boundary(O.DOMINO, steps))
    return T.Domain.from_boundary(T.DOMINO, steps), st, O.DOMINO, dict(scalar=0x6A09E667)


@pytest.mark.parametrize("random_order", [False, True])
@pytest.mark.parametrize("name", ["aztec_half", "aztec_site", "hexagon", "dwbc", "region_U"])
def test_resume_equals_uninterrupted(T, name, random_order):
    dom, st0, lat, thr = _case(T, name)
    if "t16" in thr:
        th, okw = T.thresholds(table16=thr["t16"]), dict(t16=thr["t16"])
    elif "site" in thr:
        th, okw = T.thresholds(site=thr["site"]), dict(t_site=thr["site"])
    else:
        th, okw = T.thresholds(scalar=thr["scalar"]), dict(t_scalar=thr["scalar"])
    k = 37
    ctx = T.Context(0)
    a = T.Chain(ctx, dom, seed=12, stream_id=3, th=th, init=st0)
    b = T.Chain(ctx, dom, seed=12, stream_id=3, th=th, init=st0)
    if random_order:
        a.set_order(True)
        b.set_order(True)
    a.run(2 * k)
    b.run(k)
    blob = b.checkpoint()
    b.close()
    ctx2 = T.Context(0)
    r = T.Chain.restore(ctx2, blob, dom)
    assert r.sweep == k
    r.run(k)
    assert r.sweep == 2 * k
    assert r.state_hash() == a.state_hash()
    got = r.read_state()
    assert np.array_equal(got, a.read_state())
    st = st0.copy()
    O.sweeps(lat, st, seed=12, stream=3, k=2 * k, random_order=random_order, **okw)
    assert np.array_equal(got, st)
    # the restored chain keeps the start: reset goes back to it
    r.reset()
    assert np.array_equal(r.read_state(), st0)
    # a checkpoint restores into the same context too, and twice
    r2 = T.Chain.restore(ctx, blob, dom)
    r3 = T.Chain.restore(ctx, blob, dom)
    r2.run(5)
    r3.run(5)
    assert r2.state_hash() == r3.state_hash()


def test_restore_rejects_bad_blobs(T):
    ctx = T.Context(0)
    ch = T.Chain(ctx, T.Domain.aztec(10), seed=1, th=T.thresholds(scalar=1 << 31))
    blob = bytearray(ch.checkpoint())
    for bad in (b"", bytes(blob[:20]), b"XXXX" + bytes(blob[4:]), bytes(blob[:-1])):
        with pytest.raises(T.TilingError) as e:
            T.Chain.restore(ctx, bad)
        assert e.value.code == T.TL_EINVAL
    # a state that is not a tiling of the domain is refused
    tampered = bytearray(blob)
    tampered[-5] ^= 1
    with pytest.raises(T.TilingError) as e:
        T.Chain.restore(ctx, bytes(tampered))
    assert e.value.code == T.TL_EINVAL


def test_context_sm_limit_keeps_results(T):
    # a context limited to 40 SMs plans fewer stripes; the chain is the same
    full = T.Context(0)
    small = T.Context(0, max_sms=40)
    dom = T.Domain.aztec(1500)
    a = T.Chain(full, dom, seed=3, th=T.thresholds(scalar=1 << 31))
    b = T.Chain(small, dom, seed=3, th=T.thresholds(scalar=1 << 31))
    assert b.plan()["ctas"] <= 40 < a.plan()["ctas"]
    a.run(50)
    b.run(50)
    assert a.state_hash() == b.state_hash()
