"""GPU parity on domains given by a boundary path, and coupling from the past.

Domains from a closed lattice path (Sec. 1.1) may have rows made of several
runs of sites; the sweeps and the height integration must handle them.  The
oracle builds the region from the same path by itself and finds a tiling by
search; the chain starts from that tiling on both sides.

Coupling from the past (Sec. 1.1.4): the library's exact sample and the
number of sweeps it needed must equal the oracle's, which runs the same
negative-time schedule from its own extreme tilings.
"""
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


def _comb(width, tooth, gap, teeth, base):
    """Domino path of a comb: a base of `base` rows and `teeth` teeth of width
    `tooth` and height `gap`... every row above the base holds many runs."""
    steps = [0] * width + [1] * base
    x = width
    pitch = (width - tooth) // max(teeth - 1, 1)
    for i in range(teeth):
        xr = width - i * pitch          # right edge of tooth i
        steps += [2] * (x - xr)         # along the top of the base (or nothing)
        steps += [1] * gap + [2] * tooth + [3] * gap
        x = xr - tooth
    steps += [2] * x + [3] * base
    return steps


DOMINO_PATHS = {
    "comb": lambda: _comb(width=300, tooth=6, gap=21, teeth=12, base=10),
    "U": lambda: [0] * 290 + [1] * 40 + [2] * 40 + [3] * 30 + [2] * 210 + [1] * 30 + [2] * 40 + [3] * 40,
}


@pytest.mark.parametrize("name", sorted(DOMINO_PATHS))
@pytest.mark.parametrize("kernel", [1, 2])
def test_domino_region_parity(T, ctx, name, kernel):
    steps = DOMINO_PATHS[name]()
    reg = O.region_from_boundary(O.DOMINO, steps)
    st = O.tiling_by_search(O.DOMINO, reg)
    assert st is not None
    dom = T.Domain.from_boundary(T.DOMINO, steps)
    ch = T.Chain(ctx, dom, seed=21, stream_id=4, th=T.thresholds(scalar=0x6A09E667), init=st)
    ch.set_plan(kernel)
    ring = ch.run_hashed(25)
    ohash = O.sweeps(O.DOMINO, st, seed=21, stream=4, k=25, t_scalar=0x6A09E667, want_hashes=True)
    assert np.array_equal(ring, ohash)
    assert np.array_equal(ch.read_state(), st)
    h, bad = O.height(O.DOMINO, st)
    assert bad == 0
    assert np.array_equal(ch.read_height(), h)


def test_lozenge_region_parity(T, ctx):
    # a large hexagon with a rectangular notch cut into its upper side
    a, b, c = 150, 60, 70
    steps = [0] * a + [2] * b + [1] * c + [3] * 40 + [4] * 30 + [3] * 30 + [1] * 30 + [3] * (a - 70) \
        + [5] * b + [4] * c
    reg = O.region_from_boundary(O.LOZENGE, steps)
    st = O.tiling_by_search(O.LOZENGE, reg)
    assert st is not None
    dom = T.Domain.from_boundary(T.LOZENGE, steps)
    ta, _ = O.lozenge_thresholds(0.97)
    ch = T.Chain(ctx, dom, seed=5, stream_id=2, th=T.thresholds(scalar=ta), init=st)
    ring = ch.run_hashed(20)
    ohash = O.sweeps(O.LOZENGE, st, seed=5, stream=2, k=20, t_scalar=ta, want_hashes=True)
    assert np.array_equal(ring, ohash)
    h, bad = O.height(O.LOZENGE, st)
    assert bad == 0
    assert np.array_equal(ch.read_height(), h)


@pytest.mark.parametrize("case", ["aztec10", "aztec17", "hex546", "dwbc9", "region_U"])
def test_cftp_matches_oracle(T, ctx, case):
    if case.startswith("aztec"):
        n = int(case[5:])
        dom, st0, lat = T.Domain.aztec(n), O.aztec(n), O.DOMINO
        th, okw = T.thresholds(scalar=1 << 31), dict(t_scalar=1 << 31)
    elif case == "hex546":
        dom, st0, lat = T.Domain.hexagon(5, 4, 6), O.hexagon(5, 4, 6), O.LOZENGE
        ta, _ = O.lozenge_thresholds(0.8)
        th, okw = T.thresholds(scalar=ta), dict(t_scalar=ta)
    elif case == "dwbc9":
        dom, st0, lat = T.Domain.dwbc(9), O.dwbc(9), O.SIXV
        t16 = O.sixv_thresholds(SQ2)
        th, okw = T.thresholds(table16=t16), dict(t16=t16)
    else:
        steps = [0] * 12 + [1] * 10 + [2] * 4 + [3] * 6 + [2] * 4 + [1] * 6 + [2] * 4 + [3] * 10
        reg = O.region_from_boundary(O.DOMINO, steps)
        st0, lat = O.tiling_by_search(O.DOMINO, reg), O.DOMINO
        dom = T.Domain.from_boundary(T.DOMINO, steps)
        th, okw = T.thresholds(scalar=0x50000000), dict(t_scalar=0x50000000)
    top, bot = O.extreme(lat, st0, True), O.extreme(lat, st0, False)
    want, T_o = O.cftp(lat, top, bot, seed=77, stream=3, t0=4, **okw)
    got, T_g = T.cftp(ctx, dom, seed=77, stream_id=3, th=th, t0=4)
    assert T_g == T_o
    assert np.array_equal(got, want)


def test_cftp_gives_up_at_tmax(T, ctx):
    dom = T.Domain.aztec(30)
    with pytest.raises(T.TilingError) as e:
        T.cftp(ctx, dom, seed=1, th=T.thresholds(scalar=1 << 31), t0=1, tmax=4)
    assert e.value.code == T.TL_EBUDGET


@pytest.mark.parametrize("kernel", [1, 2])
def test_volume_weighted_domino_parity(T, ctx, kernel):
    # volume weights q = 20 on black vertices (x + y even) and 1/20 on white
    # ones, and random ones (Sec. 1.1.1), per-site thresholds on both paths
    n = 70
    st = O.aztec(n)
    yy, xx = np.mgrid[0:2 * n + 1, 0:2 * n + 1]
    for q in (np.where((xx + yy) % 2 == 0, 20.0, 1 / 20.0),
              np.exp(0.3 * np.random.default_rng(2).standard_normal(xx.shape))):
        dom = T.Domain.aztec(n)
        t = dom.volume_thresholds(q)
        assert np.array_equal(t, O.volume_thresholds(O.DOMINO, q))
        ch = T.Chain(ctx, dom, seed=13, stream_id=1, th=T.thresholds(site=t))
        ch.set_plan(kernel)
        s = st.copy()
        ring = ch.run_hashed(30)
        ohash = O.sweeps(O.DOMINO, s, seed=13, stream=1, k=30, t_site=t, want_hashes=True)
        assert np.array_equal(ring, ohash)
        assert np.array_equal(ch.read_state(), s)


def test_cftp_volume_weighted_matches_oracle(T, ctx):
    n = 9
    dom, st0 = T.Domain.aztec(n), O.aztec(n)
    q = np.exp(0.5 * np.random.default_rng(4).standard_normal(st0.shape[1:]))
    t = O.volume_thresholds(O.DOMINO, q)
    top, bot = O.extreme(O.DOMINO, st0, True), O.extreme(O.DOMINO, st0, False)
    want, T_o = O.cftp(O.DOMINO, top, bot, seed=31, stream=0, t0=4, t_site=t)
    got, T_g = T.cftp(ctx, dom, seed=31, th=T.thresholds(site=t), t0=4)
    assert T_g == T_o and np.array_equal(got, want)


@pytest.mark.parametrize("kernel,halo", [(1, 0), (2, 0), (2, 3), (2, 5)])
@pytest.mark.parametrize("kind", ["aztec", "aztec_t", "hex", "dwbc"])
def test_random_order_parity(T, ctx, kind, kernel, halo):
    # random colour per pass slot (RandomWalk, Sec. 2.2) on both paths
    if kind.startswith("aztec"):
        dom, st, lat = T.Domain.aztec(90), O.aztec(90), O.DOMINO
        t = (1 << 31) if kind == "aztec" else 0x5A000000
        th, okw = T.thresholds(scalar=t), dict(t_scalar=t)
    elif kind == "hex":
        dom, st, lat = T.Domain.hexagon(60, 70, 50), O.hexagon(60, 70, 50), O.LOZENGE
        ta, _ = O.lozenge_thresholds(1.1)
        th, okw = T.thresholds(scalar=ta), dict(t_scalar=ta)
    else:
        dom, st, lat = T.Domain.dwbc(150), O.dwbc(150), O.SIXV
        t16 = O.sixv_thresholds(SQ2)
        th, okw = T.thresholds(table16=t16), dict(t16=t16)
    ch = T.Chain(ctx, dom, seed=101, stream_id=6, th=th)
    ch.set_plan(kernel, 0, halo)
    ch.set_order(True)
    ring = ch.run_hashed(24)
    ohash = O.sweeps(lat, st, seed=101, stream=6, k=24, random_order=True, want_hashes=True, **okw)
    assert np.array_equal(ring, ohash)
    assert np.array_equal(ch.read_state(), st)


def test_random_order_chain_cannot_join_a_batch(T, ctx):
    ch = T.Chain(ctx, T.Domain.aztec(20), seed=1, th=T.thresholds(scalar=1 << 31))
    ch.set_order(True)
    with pytest.raises(T.TilingError) as e:
        T.Batch(ctx, [ch])
    assert e.value.code == T.TL_EUNSUPPORTED
