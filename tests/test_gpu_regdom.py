"""GPU parity of the register-resident domino kernel (plan kernel 3).

Dominoes at t = 2^31 (each rotatable site goes UP with probability 1/2,
Sec. 1.1.3) run by default on a kernel that keeps every 128-site group of two
rows in one thread's registers for a whole launch and exchanges boundary
rows between stripes every `halo` passes.  Its result must equal the
oracle's after every sweep, whatever the halo, the launch split, the pass
order or the shape of the domain (rows made of several runs of sites, domains
narrower and wider than one stripe's threads).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from tests.test_gpu_regions_cftp import DOMINO_PATHS

pytestmark = pytest.mark.gpu

T_HALF = 1 << 31


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


def _run(T, ctx, dom, st, *, seed, stream=0, k, halo=0, spl=0, random_order=False, kernel=3):
    ch = T.Chain(ctx, dom, seed=seed, stream_id=stream, th=T.thresholds(scalar=T_HALF), init=st.copy())
    if random_order:
        ch.set_order(True)
    ch.set_plan(kernel, spl, halo)
    plan = ch.plan()
    ring = ch.run_hashed(k)
    want = st.copy()
    ohash = O.sweeps(O.DOMINO, want, seed=seed, stream=stream, k=k, t_scalar=T_HALF, want_hashes=True,
                     random_order=random_order)
    bad = np.nonzero(ring != ohash)[0]
    assert bad.size == 0, "first mismatch at sweep %d (plan %s)" % (bad[0], plan)
    got = ch.read_state()
    assert np.array_equal(got, want)
    assert ch.state_hash() == O.state_hash(want)
    return ch, want, plan


@pytest.mark.parametrize("halo", [2, 4, 6, 8, 12, 16])
@pytest.mark.parametrize("n", [40, 129, 300])
def test_aztec_halos(T, ctx, n, halo):
    ch, _, plan = _run(T, ctx, T.Domain.aztec(n), O.aztec(n), seed=23, stream=1, k=40, halo=halo)
    assert plan["kernel"] == 3 and plan["halo"] == halo


@pytest.mark.parametrize("wh", [(2, 2), (300, 7), (255, 8), (7, 40), (64, 64), (1000, 30), (30, 1000)])
def test_rectangles(T, ctx, wh):
    w, h = wh
    try:
        _run(T, ctx, T.Domain.rect(w, h), O.rect(w, h), seed=12345, stream=3, k=50, halo=2)
    except T.TilingError as e:
        # too few row pairs for two stripes with this halo is the only refusal
        assert e.code == T.TL_EUNSUPPORTED, e


@pytest.mark.parametrize("name", sorted(DOMINO_PATHS))
@pytest.mark.parametrize("halo", [2, 6])
def test_regions(T, ctx, name, halo):
    steps = DOMINO_PATHS[name]()
    st = O.tiling_by_search(O.DOMINO, O.region_from_boundary(O.DOMINO, steps))
    assert st is not None
    dom = T.Domain.from_boundary(T.DOMINO, steps)
    _run(T, ctx, dom, st, seed=21, stream=4, k=60, halo=halo)


def test_from_exact_sample(T, ctx):
    # a disordered start (an exact sample) exercises every flip pattern at once
    n = 200
    st = O.aztec_shuffle(n, 3, stream=0)
    _run(T, ctx, T.Domain.aztec(n), st, seed=8, stream=2, k=80, halo=8)


@pytest.mark.parametrize("halo", [2, 8])
def test_random_pass_order(T, ctx, halo):
    _run(T, ctx, T.Domain.aztec(150), O.aztec(150), seed=5, stream=7, k=60, halo=halo, random_order=True)


@pytest.mark.parametrize("spl", [1, 3, 7])
def test_launch_splits(T, ctx, spl):
    _run(T, ctx, T.Domain.aztec(128), O.aztec(128), seed=31, k=30, halo=6, spl=spl)


def test_default_plan_is_register_resident(T, ctx):
    ch = T.Chain(ctx, T.Domain.aztec(2048), seed=7, th=T.thresholds(scalar=T_HALF))
    plan = ch.plan()
    assert plan["kernel"] == 3, plan
    # other thresholds take one of the general kernels
    ch2 = T.Chain(ctx, T.Domain.aztec(2048), seed=7, th=T.thresholds(scalar=0x7FFFFFFF))
    assert ch2.plan()["kernel"] in (1, 2)


def test_density_and_nsew(T, ctx):
    n = 90
    dom = T.Domain.aztec(n)
    ch = T.Chain(ctx, dom, seed=4, th=T.thresholds(scalar=T_HALF))
    ch.set_plan(3, 0, 4)
    ch.density_begin(stride=3, burn_in=10)
    ch.run(17)
    ch.run(40)
    dens, samples = ch.read_density()
    st = O.aztec(n)
    counts = np.zeros(st.shape, dtype=np.uint32)
    ncounts = np.zeros((4, 2 * n, 2 * n), dtype=np.uint32)
    nsamp = 0
    for s in range(57):
        O.sweeps(O.DOMINO, st, seed=4, sweep0=s, k=1, t_scalar=T_HALF)
        if s + 1 >= 10 and (s + 1 - 10) % 3 == 0:
            O.accumulate(st, counts)
            O.domino_nsew(st, n % 2, ncounts)
            nsamp += 1
    assert samples == nsamp
    assert np.array_equal(np.rint(dens * nsamp).astype(np.uint32), counts)
    assert np.array_equal(np.rint(ch.read_nsew() * nsamp).astype(np.uint32), ncounts)


@pytest.mark.parametrize("shape,halo,min_threads", [(("aztec", 100), 0, 0), (("aztec", 129), 4, 0),
                                                    (("rect", 9000, 30), 8, 385)])
def test_density_many_samples(T, ctx, shape, halo, min_threads):
    # a sample after every sweep for 300 sweeps, so the bit-sliced counters
    # carry through nine planes; both ways the kernel adds a pair's blocks
    # (all eight at once, or row by row in the 512-thread build) and the
    # odd last vertex row of the box must count exactly what the oracle does
    if shape[0] == "aztec":
        dom, st = T.Domain.aztec(shape[1]), O.aztec(shape[1])
    else:
        dom, st = T.Domain.rect(shape[1], shape[2]), O.rect(shape[1], shape[2])
    ch = T.Chain(ctx, dom, seed=6, th=T.thresholds(scalar=T_HALF), init=st.copy())
    ch.set_plan(3, 0, halo)
    plan = ch.plan()
    assert plan["kernel"] == 3 and plan["threads"] >= min_threads, plan
    ch.density_begin(stride=1, burn_in=0)
    ch.run(300)
    dens, samples = ch.read_density()
    counts = np.zeros(st.shape, dtype=np.uint32)
    for s in range(300):
        O.sweeps(O.DOMINO, st, seed=6, sweep0=s, k=1, t_scalar=T_HALF)
        O.accumulate(st, counts)
    assert samples == 300
    assert np.array_equal(np.rint(dens * 300).astype(np.uint32), counts)
    assert np.array_equal(ch.read_state(), st)


def test_kernels_agree_at_full_size(T, ctx):
    # the register-resident and the shared-memory resident kernels give the
    # same chain on the benchmark domain (Aztec 2048), 300 sweeps
    dom = T.Domain.aztec(2048)
    a = T.Chain(ctx, dom, seed=7, th=T.thresholds(scalar=T_HALF))
    b = T.Chain(ctx, dom, seed=7, th=T.thresholds(scalar=T_HALF))
    a.set_plan(3)
    b.set_plan(2)
    ra = a.run_hashed(300)
    rb = b.run_hashed(300)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.read_state(), b.read_state())
