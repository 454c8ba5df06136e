"""Host-side checks of the C-ABI library (no GPU needed).

The library must load and export every function declared in include/tiling.h;
its host-side domain builders and FP64 threshold builders must agree bit for
bit with the independent oracle.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1804_07250_gb300 as T
    return T


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "tiling.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tl_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(T):
    names = _declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(T.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(T.EXPORTED) <= set(names)
    assert "sm_103a" in T.version()


@pytest.mark.parametrize("n", [1, 2, 5, 32])
def test_aztec_domain_matches_oracle(T, n):
    d = T.Domain.aztec(n)
    assert np.array_equal(d.initial_state(), O.aztec(n))
    assert d.info.sites == n * n + (n - 1) * (n - 1)
    assert d.info.edges == 4 * n * n
    assert d.info.passes == 2 and d.info.planes == 2


@pytest.mark.parametrize("w,h", [(4, 4), (5, 4), (6, 3), (10, 7)])
def test_rect_domain_matches_oracle(T, w, h):
    d = T.Domain.rect(w, h)
    assert np.array_equal(d.initial_state(), O.rect(w, h))
    assert d.info.sites == (w - 1) * (h - 1)


def test_rect_untileable(T):
    with pytest.raises(T.TilingError) as e:
        T.Domain.rect(3, 5)
    assert e.value.code == T.TL_ENOTTILEABLE


@pytest.mark.parametrize("abc", [(1, 1, 1), (2, 3, 4), (5, 2, 3), (16, 16, 16)])
def test_hexagon_domain_matches_oracle(T, abc):
    a, b, c = abc
    d = T.Domain.hexagon(a, b, c)
    assert np.array_equal(d.initial_state(), O.hexagon(a, b, c))
    # interior vertices of the hexagon: ab + bc + ca - (a + b + c) + 1
    assert d.info.sites == a * b + b * c + c * a - (a + b + c) + 1
    assert d.info.passes == 3 and d.info.planes == 3


@pytest.mark.parametrize("N", [2, 3, 7, 64])
def test_dwbc_domain_matches_oracle(T, N):
    d = T.Domain.dwbc(N)
    assert np.array_equal(d.initial_state(), O.dwbc(N))
    assert d.info.sites == (N - 1) ** 2
    assert d.info.edges == 2 * N * (N - 1)
    assert d.info.passes == 4


def test_large_domain_sizes(T):
    d = T.Domain.aztec(2048)
    assert d.info.sites == 8_384_513
    assert d.info.width == 4097
    d = T.Domain.hexagon(1024, 1024, 1024)
    assert d.info.sites == 3_142_657
    d = T.Domain.dwbc(2048)
    assert d.info.sites == 4_190_209


def test_bad_sizes_rejected(T):
    for fn, args in [(T.Domain.aztec, (0,)), (T.Domain.aztec, (40000,)),
                     (T.Domain.hexagon, (0, 1, 1)), (T.Domain.dwbc, (1,)),
                     (T.Domain.rect, (0, 4))]:
        with pytest.raises(T.TilingError) as e:
            fn(*args)
        assert e.value.code == T.TL_EINVAL


def test_domino_thresholds_bit_exact(T):
    d = T.Domain.aztec(7)
    rng = np.random.default_rng(0)
    w = np.exp(0.5 * rng.standard_normal((2, 15, 15)))
    assert np.array_equal(d.domino_thresholds(w), O.domino_thresholds(w))
    assert np.all(d.domino_thresholds(np.ones((2, 15, 15))) == 1 << 31)
    with pytest.raises(T.TilingError):
        d.domino_thresholds(-w)


@pytest.mark.parametrize("q", [0.9995, 0.5, 1.0, 3.0, 1e-6])
def test_lozenge_thresholds_bit_exact(T, q):
    assert T.lozenge_thresholds(q) == O.lozenge_thresholds(q)


def test_sixv_thresholds_bit_exact(T):
    rng = np.random.default_rng(3)
    for w6 in [[1, 1, 1, 1, math.sqrt(2), math.sqrt(2)], [1] * 6,
               [1, 1, 1, 1, math.sqrt(8), math.sqrt(8)]] + [list(rng.uniform(0.1, 3, 6)) for _ in range(20)]:
        assert np.array_equal(T.sixv_thresholds(w6), O.sixv_thresholds(w6))
    with pytest.raises(T.TilingError):
        T.sixv_thresholds([1, 1, 0, 1, 1, 1])


# ---------------------------------------------------------------------------
# Extreme configurations and domains from a boundary path (host code)
# ---------------------------------------------------------------------------
def _builtin(T, kind, args):
    dom = {"aztec": T.Domain.aztec, "rect": T.Domain.rect, "hex": T.Domain.hexagon,
           "dwbc": T.Domain.dwbc}[kind](*args)
    st = {"aztec": O.aztec, "rect": O.rect, "hex": O.hexagon, "dwbc": O.dwbc}[kind](*args)
    lat = {"aztec": O.DOMINO, "rect": O.DOMINO, "hex": O.LOZENGE, "dwbc": O.SIXV}[kind]
    return dom, st, lat


@pytest.mark.parametrize("kind,args", [("aztec", (1,)), ("aztec", (2,)), ("aztec", (5,)), ("aztec", (12,)),
                                       ("rect", (6, 5)), ("rect", (7, 4)), ("hex", (1, 1, 1)),
                                       ("hex", (3, 5, 4)), ("hex", (6, 2, 7)), ("dwbc", (2,)),
                                       ("dwbc", (7,)), ("dwbc", (16,))])
def test_extreme_states_match_oracle(T, kind, args):
    # Thurston's extreme tilings (host, product) against the oracle's pointwise
    # height pushes from its own starting tiling
    dom, st, lat = _builtin(T, kind, args)
    assert np.array_equal(dom.extreme_state("top"), O.extreme(lat, st, True))
    assert np.array_equal(dom.extreme_state("bottom"), O.extreme(lat, st, False))


def _shapes():
    sys_path = os.path.join(ROOT, "tests")
    import sys
    if sys_path not in sys.path:
        sys.path.insert(0, sys_path)
    from test_oracle_pins import DOMINO_SHAPES, _aztec_path
    shapes = dict(DOMINO_SHAPES)
    shapes["aztec9"] = _aztec_path(9)
    # a spiral corridor of width 2 (many segments per row)
    shapes["zigzag"] = ([0] * 8 + [1] * 2 + [2] * 6 + [1] * 2 + [0] * 6 + [1] * 2 + [2] * 8 + [3] * 6)
    return shapes


@pytest.mark.parametrize("name", ["square4", "L", "U", "aztec4", "aztec9", "zigzag"])
def test_domino_from_boundary_matches_oracle(T, name):
    steps = _shapes()[name]
    reg = O.region_from_boundary(O.DOMINO, steps)
    dom = T.Domain.from_boundary(T.DOMINO, steps)
    face, W, H = reg
    assert dom.canon_shape == (2, H, W)
    ost = O.tiling_by_search(O.DOMINO, reg)
    assert np.array_equal(dom.initial_state(), O.extreme(O.DOMINO, ost, False))
    assert np.array_equal(dom.extreme_state("top"), O.extreme(O.DOMINO, ost, True))


def test_aztec_boundary_gives_the_aztec_domain(T):
    _shapes()   # puts tests/ on the path
    from test_oracle_pins import _aztec_path
    for n in (3, 8):
        dom = T.Domain.from_boundary(T.DOMINO, _aztec_path(n))
        ref = T.Domain.aztec(n)
        assert dom.info.sites == ref.info.sites and dom.info.edges == ref.info.edges
        assert np.array_equal(dom.initial_state(), ref.extreme_state("bottom"))


LOZENGE_SHAPES = {
    "hex213": [0] * 2 + [2] * 1 + [1] * 3 + [3] * 2 + [5] * 1 + [4] * 3,
    "hex444": [0] * 4 + [2] * 4 + [1] * 4 + [3] * 4 + [5] * 4 + [4] * 4,
    # hexagon with a notch: non-convex rows
    "notched": [0] * 4 + [2] * 2 + [1] * 3 + [3] * 1 + [4] * 1 + [3] * 1 + [1] * 1 + [3] * 2
               + [5] * 2 + [4] * 3,
}


@pytest.mark.parametrize("name", sorted(LOZENGE_SHAPES))
def test_lozenge_from_boundary_matches_oracle(T, name):
    steps = LOZENGE_SHAPES[name]
    reg = O.region_from_boundary(O.LOZENGE, steps)
    ost = O.tiling_by_search(O.LOZENGE, reg)
    if ost is None:
        with pytest.raises(T.TilingError) as e:
            T.Domain.from_boundary(T.LOZENGE, steps)
        assert e.value.code == T.TL_ENOTTILEABLE
        return
    dom = T.Domain.from_boundary(T.LOZENGE, steps)
    assert np.array_equal(dom.initial_state(), O.extreme(O.LOZENGE, ost, False))
    assert np.array_equal(dom.extreme_state("top"), O.extreme(O.LOZENGE, ost, True))


def test_from_boundary_errors(T):
    cases = [
        (T.DOMINO, [0] * 3 + [1] * 3 + [2] * 3 + [3] * 3, T.TL_ENOTTILEABLE),        # odd area
        (T.DOMINO, [0] * 3 + [1] * 3 + [2] + [1] + [2] * 3 + [3] * 3 + [0] + [3],
         T.TL_ENOTTILEABLE),                                                     # two opposite corners cut
        (T.DOMINO, [0, 0, 1, 1, 2, 2], T.TL_EINVAL),                                # not closed
        (T.DOMINO, [0, 0, 1, 2, 3, 2, 1, 1, 0, 3, 3, 2], T.TL_ENOTSIMPLY),          # revisits a point
        (T.DOMINO, [0, 5, 2, 3], T.TL_EINVAL),                                      # bad step code
        (T.SIXV, [0, 1, 2, 3], T.TL_EINVAL),                                        # lattice without paths
    ]
    for lat, steps, code in cases:
        with pytest.raises(T.TilingError) as e:
            T.Domain.from_boundary(lat, steps)
        assert e.value.code == code, (steps, e.value)


@pytest.mark.parametrize("kind,args", [("aztec", (9,)), ("rect", (8, 5)), ("hex", (4, 3, 5))])
def test_volume_thresholds_bit_exact(T, kind, args):
    dom, st, lat = _builtin(T, kind, args)
    rng = np.random.default_rng(17)
    q = np.exp(0.8 * rng.standard_normal(st.shape[1:]))
    q[0, 0] = 1e-70            # extreme weights round to 0 / clamp to 2^32 - 1
    q[-1, -1] = 1e70
    assert np.array_equal(dom.volume_thresholds(q), O.volume_thresholds(lat, q))
    for bad in (-q, q * 0 + 1e80):
        with pytest.raises(T.TilingError):
            dom.volume_thresholds(bad)
