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
