"""Domino shuffling on the GPU, and the arctic circle.

The library's shuffling sampler must give exactly the oracle's tiling for the
same seed and stream.  Its exact samples of large Aztec diamonds, and the
Markov chain started from one and from the all-horizontal tiling, must show
the arctic circle: the four frozen corners (brickwork of one domino type)
fill 1 - pi/4 of the diamond, outside the inscribed circle of radius n/sqrt 2.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


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


def _aztec_faces(n):
    c = np.arange(2 * n) + 0.5 - n
    return (np.abs(c)[None, :] + np.abs(c)[:, None]) <= n


def face_types(st, n):
    """Per face (lower-left corner (x, y) of the box): 0 N, 1 S, 2 E, 3 W,
    -1 off the diamond.  A horizontal domino is north iff its left square has
    colour (x + y) mod 2 == n mod 2; a vertical one is west iff its bottom
    square's colour differs from n mod 2."""
    kappa = n % 2
    W = 2 * n + 1
    t = np.full((W - 1, W - 1), -1, dtype=np.int8)
    ys, xs = np.nonzero(st[1])              # Vt(x, y): horizontal domino on (x-1, y), (x, y)
    kind = np.where((xs - 1 + ys) % 2 == kappa, 0, 1).astype(np.int8)
    t[ys, xs - 1] = kind
    t[ys, xs] = kind
    ys, xs = np.nonzero(st[0])              # Hz(x, y): vertical domino on (x, y-1), (x, y)
    kind = np.where((xs + ys - 1) % 2 != kappa, 3, 2).astype(np.int8)
    t[ys - 1, xs] = kind
    t[ys, xs] = kind
    return t


def frozen_fraction(st, n, win=16, level=0.98):
    """Fraction of the diamond's faces whose centred win x win window is at
    least `level` one type (faces off the diamond are not counted)."""
    from scipy.ndimage import uniform_filter
    t = face_types(st, n)
    inside = t >= 0
    cnt = uniform_filter(inside.astype(np.float64), size=win, mode="constant")
    best = np.zeros_like(cnt)
    for k in range(4):
        best = np.maximum(best, uniform_filter((t == k).astype(np.float64), size=win, mode="constant"))
    frac = np.where(cnt > 0, best / np.maximum(cnt, 1e-12), 0)
    return float(((frac >= level) & inside).sum() / inside.sum()), t


@pytest.mark.parametrize("n,seed,stream", [(1, 0, 0), (2, 5, 1), (3, 2, 0), (7, 11, 2), (40, 3, 9), (129, 8, 4),
                                           (201, 6, 7)])
def test_shuffle_matches_oracle(T, ctx, n, seed, stream):
    got = T.aztec_shuffle(ctx, n, seed=seed, stream_id=stream)
    want = O.aztec_shuffle(n, seed, stream)
    assert np.array_equal(got, want)


def test_shuffle_graph_reused_across_seeds_and_orders(T, ctx):
    # the context keeps one graph per order: same order with new seeds, and
    # a change of order and back, all still match the oracle
    for n, seed, stream in [(40, 1, 0), (40, 2, 0), (40, 2, 5), (7, 3, 1), (40, 4, 2)]:
        got = T.aztec_shuffle(ctx, n, seed=seed, stream_id=stream)
        assert np.array_equal(got, O.aztec_shuffle(n, seed, stream))


def test_shuffle_large_is_a_tiling_with_the_arctic_circle(T, ctx):
    n = 2048
    st = T.aztec_shuffle(ctx, n, seed=2024, stream_id=0)
    assert O.domino_check(st, _aztec_faces(n)) == 0
    h, bad = O.height(O.DOMINO, st)
    assert bad == 0
    ff, t = frozen_fraction(st, n)
    assert abs(ff - (1 - math.pi / 4)) < 0.02, ff
    # the top cap (beyond 1.05 n / sqrt 2 from the centre, above it) is north brickwork
    c = np.arange(2 * n) + 0.5 - n
    X, Y = np.meshgrid(c, c)
    cap = (t >= 0) & (np.hypot(X, Y) > 1.05 * n / math.sqrt(2)) & (Y > np.abs(X))
    assert (t[cap] == 0).mean() >= 0.98
    # the frozen boundary crosses the vertical axis near n / sqrt 2
    col = t[:, n]                                    # faces just right of the axis
    ys = c[(col != 0) & (col >= 0)]
    top_disorder = ys.max()                          # highest non-north face on the axis
    assert abs(top_disorder - n / math.sqrt(2)) < 0.02 * n + 16


def test_glauber_keeps_the_exact_law_and_reaches_it(T, ctx):
    # started from an exact sample, the chain stays at the arctic shape;
    # started from all-horizontal it reaches it after O(n^2) sweeps
    n = 256
    exact = T.aztec_shuffle(ctx, n, seed=7)
    ff_exact, _ = frozen_fraction(exact, n)
    dom = T.Domain.aztec(n)
    ch = T.Chain(ctx, dom, seed=99, th=T.thresholds(scalar=1 << 31), init=exact)
    ch.run(4000)
    ff_chain, _ = frozen_fraction(ch.read_state(), n)
    assert abs(ff_chain - ff_exact) < 0.03, (ff_chain, ff_exact)
    ch2 = T.Chain(ctx, dom, seed=98, th=T.thresholds(scalar=1 << 31))
    ch2.run(6 * n * n)
    ff_burn, _ = frozen_fraction(ch2.read_state(), n)
    assert abs(ff_burn - ff_exact) < 0.03, (ff_burn, ff_exact)


def test_chain_reaches_the_arctic_circle_at_order_1024(T, ctx):
    # the heat-bath chain itself (t = 2^31), from the all-horizontal tiling,
    # after 6 n^2 sweeps: frozen fraction within 0.02 of 1 - pi/4, north
    # brickwork in the top cap, the frozen boundary crossing the vertical
    # axis near n / sqrt 2
    n = 1024
    dom = T.Domain.aztec(n)
    ch = T.Chain(ctx, dom, seed=2025, stream_id=1, th=T.thresholds(scalar=1 << 31))
    ch.run(6 * n * n)
    st = ch.read_state()
    assert O.domino_check(st, _aztec_faces(n)) == 0
    ff, t = frozen_fraction(st, n)
    assert abs(ff - (1 - math.pi / 4)) < 0.02, ff
    c = np.arange(2 * n) + 0.5 - n
    X, Y = np.meshgrid(c, c)
    cap = (t >= 0) & (np.hypot(X, Y) > 1.05 * n / math.sqrt(2)) & (Y > np.abs(X))
    assert (t[cap] == 0).mean() >= 0.98
    col = t[:, n]
    ys = c[(col != 0) & (col >= 0)]
    assert abs(ys.max() - n / math.sqrt(2)) < 0.02 * n + 16
