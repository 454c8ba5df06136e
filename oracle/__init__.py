"""CPU oracle for colour-class-parallel heat-bath Glauber dynamics.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The library product never imports
this package, and this package imports nothing from the product.

Thin ctypes wrapper over ``oracle.c`` (plain single-threaded C).  Every
function documents the passage of Keating & Sridhar, "Random Tilings with the
GPU", that it follows.  States are numpy uint8 arrays in the canonical layout
``[plane, y, x]`` described in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DOMINO, LOZENGE, SIXV = "domino", "lozenge", "sixv"
PASSES = {DOMINO: 2, LOZENGE: 3, SIXV: 4}


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u8p, u32p, u64p, i32p, dp = (ctypes.c_void_p,) * 5
        c = ctypes
        sig = {
            "or_philox4x32_10": (None, [u32p, u32p, u32p]),
            "or_site_u": (c.c_uint32, [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64]),
            "or_splitmix64": (c.c_uint64, [c.c_uint64]),
            "or_slot_colour": (c.c_int, [c.c_uint64, c.c_uint32, c.c_uint32, c.c_int, c.c_int]),
            "or_state_hash": (c.c_uint64, [u8p, c.c_uint64]),
            "or_domino_aztec_init": (c.c_int, [c.c_int, u8p]),
            "or_domino_rect_init": (c.c_int, [c.c_int, c.c_int, u8p]),
            "or_domino_site_states": (None, [u8p, c.c_int, c.c_int, c.c_int, u8p]),
            "or_domino_apply_pass": (None, [u8p, c.c_int, c.c_int, c.c_int, u8p]),
            "or_domino_sweeps": (c.c_int, [u8p, c.c_int, c.c_int, u32p, c.c_uint32, c.c_uint64,
                                           c.c_uint32, c.c_uint64, c.c_uint64, u64p, c.c_int]),
            "or_domino_thresholds": (None, [dp, c.c_int, c.c_int, u32p]),
            "or_domino_weight": (c.c_double, [u8p, c.c_int, c.c_int, dp]),
            "or_domino_check": (c.c_int64, [u8p, c.c_int, c.c_int, u8p]),
            "or_domino_height": (c.c_int64, [u8p, c.c_int, c.c_int, i32p]),
            "or_lozenge_hexagon_init": (c.c_int, [c.c_int, c.c_int, c.c_int, u8p]),
            "or_lozenge_site_states": (None, [u8p, c.c_int, c.c_int, c.c_int, u8p]),
            "or_lozenge_apply_pass": (None, [u8p, c.c_int, c.c_int, c.c_int, u8p]),
            "or_lozenge_sweeps": (c.c_int, [u8p, c.c_int, c.c_int, u32p, c.c_uint32, c.c_uint64,
                                            c.c_uint32, c.c_uint64, c.c_uint64, u64p, c.c_int]),
            "or_lozenge_thresholds": (c.c_int, [c.c_double, u32p, u32p]),
            "or_lozenge_check": (c.c_int64, [u8p, c.c_int, c.c_int, u8p, u8p]),
            "or_lozenge_height": (c.c_int64, [u8p, c.c_int, c.c_int, i32p]),
            "or_sixv_dwbc_init": (c.c_int, [c.c_int, u8p]),
            "or_sixv_vertex_type": (c.c_int, [u8p, c.c_int, c.c_int, c.c_int]),
            "or_sixv_check_dwbc": (c.c_int64, [u8p, c.c_int]),
            "or_sixv_site_states": (None, [u8p, c.c_int, c.c_int, u8p]),
            "or_sixv_apply_pass": (None, [u8p, c.c_int, c.c_int, u8p]),
            "or_sixv_sweeps": (c.c_int, [u8p, c.c_int, u32p, c.c_uint64, c.c_uint32, c.c_uint64,
                                         c.c_uint64, u64p, c.c_int]),
            "or_sixv_weight": (c.c_double, [u8p, c.c_int, dp]),
            "or_sixv_thresholds": (c.c_int, [dp, u32p]),
            "or_sixv_height": (c.c_int64, [u8p, c.c_int, i32p]),
            "or_accumulate": (None, [u8p, c.c_uint64, u32p]),
            "or_domino_nsew": (None, [u8p, c.c_int, c.c_int, c.c_int, u32p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) of a 4-word counter and 2-word key."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def site_u(seed: int, stream: int, sweep: int, pass_: int, rank: int) -> int:
    """The 32-bit uniform of one site, bit-plane keyed (module docstring of oracle.c)."""
    return int(lib().or_site_u(seed, stream, sweep, pass_, rank))


def slot_colour(seed: int, stream: int, sweep: int, slot: int, passes: int) -> int:
    """Colour visited by pass slot `slot` of sweep `sweep` in random order."""
    return int(lib().or_slot_colour(seed, stream, sweep, slot, passes))


def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x))


def state_hash(st: np.ndarray) -> int:
    """Order-independent 64-bit hash of a canonical state."""
    st = np.ascontiguousarray(st, dtype=np.uint8)
    return int(lib().or_state_hash(_p(st), st.size))


# --------------------------------------------------------------------------
# Domains and initial states
# --------------------------------------------------------------------------
def aztec(n: int) -> np.ndarray:
    """Aztec diamond of order n, all-horizontal tiling; shape (2, 2n+1, 2n+1)."""
    W = 2 * n + 1
    st = np.zeros((2, W, W), dtype=np.uint8)
    lib().or_domino_aztec_init(n, _p(st))
    return st


def rect(w: int, h: int) -> np.ndarray:
    """w x h faces; all-horizontal (w even) or all-vertical (h even)."""
    st = np.zeros((2, h + 1, w + 1), dtype=np.uint8)
    if lib().or_domino_rect_init(w, h, _p(st)) != 0:
        raise ValueError("rectangle %dx%d has no domino tiling" % (w, h))
    return st


def hexagon(a: int, b: int, c: int) -> np.ndarray:
    """a x b x c hexagon, empty-box tiling; shape (3, b+c+1, a+c+1)."""
    st = np.zeros((3, b + c + 1, a + c + 1), dtype=np.uint8)
    lib().or_lozenge_hexagon_init(a, b, c, _p(st))
    return st


def dwbc(N: int) -> np.ndarray:
    """Six-vertex domain-wall boundary, identity start; shape (2, N+2, N+2)."""
    st = np.zeros((2, N + 2, N + 2), dtype=np.uint8)
    lib().or_sixv_dwbc_init(N, _p(st))
    return st


def lattice_of(st: np.ndarray, hint: str | None = None) -> str:
    if hint:
        return hint
    return LOZENGE if st.shape[0] == 3 else DOMINO


# --------------------------------------------------------------------------
# Moves
# --------------------------------------------------------------------------
def site_states(lattice: str, st: np.ndarray, pass_: int) -> np.ndarray:
    """Per site of class `pass_`: 0 not rotatable, 1 DOWN, 2 UP; shape (H, W)."""
    _, H, W = st.shape
    out = np.zeros((H, W), dtype=np.uint8)
    L = lib()
    if lattice == DOMINO:
        L.or_domino_site_states(_p(st), W, H, pass_, _p(out))
    elif lattice == LOZENGE:
        L.or_lozenge_site_states(_p(st), W, H, pass_, _p(out))
    else:
        L.or_sixv_site_states(_p(st), W - 2, pass_, _p(out))
    return out


def apply_pass(lattice: str, st: np.ndarray, pass_: int, dec: np.ndarray) -> None:
    """Cluster move on class `pass_`: rotatable sites go UP where dec=1 (in place)."""
    _, H, W = st.shape
    dec = np.ascontiguousarray(dec, dtype=np.uint8)
    L = lib()
    if lattice == DOMINO:
        L.or_domino_apply_pass(_p(st), W, H, pass_, _p(dec))
    elif lattice == LOZENGE:
        L.or_lozenge_apply_pass(_p(st), W, H, pass_, _p(dec))
    else:
        L.or_sixv_apply_pass(_p(st), W - 2, pass_, _p(dec))


def sweeps(lattice: str, st: np.ndarray, *, seed: int, stream: int = 0, sweep0: int = 0,
           k: int = 1, t_scalar: int | None = None, t_site: np.ndarray | None = None,
           t16: np.ndarray | None = None, want_hashes: bool = False, random_order: bool = False):
    """Run k heat-bath sweeps in place (Eq. 1.1 with colour-class clusters).

    Domino / lozenge: threshold t_site ([H, W] uint32) or t_scalar.  Six-vertex:
    the 16-entry table t16.  Returns the per-sweep hashes if asked.
    """
    _, H, W = st.shape
    assert st.dtype == np.uint8 and st.flags["C_CONTIGUOUS"]
    hashes = np.zeros(max(k, 1), dtype=np.uint64) if want_hashes else None
    hp = _p(hashes) if hashes is not None else None
    L = lib()
    if lattice in (DOMINO, LOZENGE):
        ts = None
        if t_site is not None:
            ts = np.ascontiguousarray(t_site, dtype=np.uint32)
            assert ts.shape == (H, W)
        tsc = 0 if t_scalar is None else int(t_scalar)
        fn = L.or_domino_sweeps if lattice == DOMINO else L.or_lozenge_sweeps
        rc = fn(_p(st), W, H, _p(ts) if ts is not None else None, tsc, seed, stream, sweep0, k, hp,
                int(random_order))
    else:
        t = np.ascontiguousarray(t16, dtype=np.uint32)
        assert t.shape == (16,)
        rc = L.or_sixv_sweeps(_p(st), W - 2, _p(t), seed, stream, sweep0, k, hp, int(random_order))
    if rc != 0:
        raise MemoryError("oracle sweep failed")
    return hashes[:k] if want_hashes else None


# --------------------------------------------------------------------------
# Thresholds and weights
# --------------------------------------------------------------------------
def domino_thresholds(w: np.ndarray) -> np.ndarray:
    """t = floor(2^32 wE wW / (wE wW + wN wS)) per vertex (Sec. 1.1.1)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    _, H, W = w.shape
    t = np.zeros((H, W), dtype=np.uint32)
    lib().or_domino_thresholds(_p(w), W, H, _p(t))
    return t


def volume_thresholds(lattice: str, q: np.ndarray) -> np.ndarray:
    """Heat-bath thresholds for volume weights (Sec. 1.1.1): the Gibbs weight
    is prod_v q_v^h(v).  A domino rotation at v moves h(v) by 4, upward for
    UP exactly when x + y is even (by the Fig. 2 rule: the block's east edge
    has the black square on its left then); a lozenge UP adds one cube.
    P(UP) = q^4 / (1 + q^4) or 1 / (1 + q^4) (dominoes), q / (1 + q)
    (lozenges); t = min(floor(2^32 P), 2^32 - 1)."""
    q = np.asarray(q, dtype=np.float64)
    H, W = q.shape
    t = np.zeros((H, W), dtype=np.uint32)
    for y in range(H):
        for x in range(W):
            qv = float(q[y, x])
            if lattice == DOMINO:
                q4 = (qv * qv) * (qv * qv)
                p = q4 / (1.0 + q4) if (x + y) % 2 == 0 else 1.0 / (1.0 + q4)
            else:
                p = qv / (1.0 + qv)
            t[y, x] = min(int(np.floor(p * 4294967296.0)), 0xFFFFFFFF)
    return t


def volume_weight(lattice: str, st: np.ndarray, q: np.ndarray) -> float:
    """prod_v q_v^h(v) over the domain's vertices (Sec. 1.1.1)."""
    h, bad = height(lattice, st)
    assert bad == 0
    m = h != HEIGHT_NONE
    return float(np.prod(np.asarray(q, dtype=np.float64)[m] ** h[m].astype(np.float64)))


def domino_weight(st: np.ndarray, w: np.ndarray) -> float:
    w = np.ascontiguousarray(w, dtype=np.float64)
    _, H, W = st.shape
    return float(lib().or_domino_weight(_p(st), W, H, _p(w)))


def lozenge_thresholds(q: float):
    ta = np.zeros(1, dtype=np.uint32)
    tr = np.zeros(1, dtype=np.uint32)
    if lib().or_lozenge_thresholds(q, _p(ta), _p(tr)) != 0:
        raise ValueError("q too small")
    return int(ta[0]), int(tr[0])


def sixv_thresholds(w6) -> np.ndarray:
    w = np.ascontiguousarray(w6, dtype=np.float64)
    t = np.zeros(16, dtype=np.uint32)
    if lib().or_sixv_thresholds(_p(w), _p(t)) != 0:
        raise ValueError("bad six-vertex table")
    return t


def sixv_weight(st: np.ndarray, w6) -> float:
    w = np.ascontiguousarray(w6, dtype=np.float64)
    return float(lib().or_sixv_weight(_p(st), st.shape[1] - 2, _p(w)))


def sixv_vertex_type(st: np.ndarray, X: int, Y: int) -> int:
    return int(lib().or_sixv_vertex_type(_p(st), st.shape[1] - 2, X, Y))


# --------------------------------------------------------------------------
# Invariants and observables
# --------------------------------------------------------------------------
def domino_check(st: np.ndarray, face_mask: np.ndarray | None = None) -> int:
    _, H, W = st.shape
    fm = None
    if face_mask is not None:
        fm = np.ascontiguousarray(face_mask, dtype=np.uint8)
        assert fm.shape == (H - 1, W - 1)
    return int(lib().or_domino_check(_p(st), W, H, _p(fm) if fm is not None else None))


def lozenge_check(st: np.ndarray, up_mask=None, dn_mask=None) -> int:
    _, H, W = st.shape
    um = np.ascontiguousarray(up_mask, dtype=np.uint8) if up_mask is not None else None
    dm = np.ascontiguousarray(dn_mask, dtype=np.uint8) if dn_mask is not None else None
    return int(lib().or_lozenge_check(_p(st), W, H, _p(um) if um is not None else None,
                                      _p(dm) if dm is not None else None))


def sixv_check_dwbc(st: np.ndarray) -> int:
    return int(lib().or_sixv_check_dwbc(_p(st), st.shape[1] - 2))


HEIGHT_NONE = np.iinfo(np.int32).min


def height(lattice: str, st: np.ndarray):
    """Height function (domino Fig. 2, lozenge cube stack, six-vertex Fig. 6).

    Returns (h, inconsistencies).  Domino / lozenge: int32 [H, W] on vertices,
    HEIGHT_NONE off the domain.  Six-vertex: int32 [N+1, N+1] on faces.
    """
    _, H, W = st.shape
    L = lib()
    if lattice == SIXV:
        N = W - 2
        h = np.zeros((N + 1, N + 1), dtype=np.int32)
        bad = L.or_sixv_height(_p(st), N, _p(h))
    else:
        h = np.zeros((H, W), dtype=np.int32)
        fn = L.or_domino_height if lattice == DOMINO else L.or_lozenge_height
        bad = fn(_p(st), W, H, _p(h))
    return h, int(bad)


def accumulate(st: np.ndarray, counts: np.ndarray) -> None:
    """Edge-occupancy counters: counts += st (uint32, same shape)."""
    assert counts.dtype == np.uint32 and counts.shape == st.shape
    lib().or_accumulate(_p(st), st.size, _p(counts))


def domino_nsew(st: np.ndarray, kappa: int, counts: np.ndarray | None = None) -> np.ndarray:
    """Per-face domino-type counters (Sec. 4's arctic-circle pictures).

    Adds one to counts[t, y, x] for both squares of every domino, t = 0 north,
    1 south, 2 east, 3 west, shape [4, H-1, W-1] (uint32).  Horizontal
    dominoes are north iff the left square's colour (x+y) mod 2 equals kappa,
    vertical ones west iff the bottom square's colour differs from kappa
    (kappa = n mod 2 for the Aztec diamond of order n).  Returns counts.
    """
    st = np.ascontiguousarray(st, dtype=np.uint8)
    _, H, W = st.shape
    if counts is None:
        counts = np.zeros((4, H - 1, W - 1), dtype=np.uint32)
    assert counts.dtype == np.uint32 and counts.shape == (4, H - 1, W - 1) and counts.flags["C_CONTIGUOUS"]
    lib().or_domino_nsew(_p(st), W, H, int(kappa), _p(counts))
    return counts


# --------------------------------------------------------------------------
# Regions from a boundary path, extreme tilings, coupling from the past
# --------------------------------------------------------------------------
_STEPS = {DOMINO: [(1, 0), (0, 1), (-1, 0), (0, -1)],
          LOZENGE: [(1, 0), (0, 1), (1, 1), (-1, 0), (0, -1), (-1, -1)]}


def _crossings(poly, W, H, offsets):
    """Winding numbers of points (x + ox, y + oy) for every lattice (x, y) and
    offset (ox, oy): the signed number of polygon edges crossing the ray from
    the point towards +x (each edge spans one row band, the path having unit
    steps).  Returns one [H, W] int array per offset."""
    out = []
    for ox, oy in offsets:
        cnt = np.zeros((H, W + 1), dtype=np.int64)
        n = len(poly)
        for i in range(n):
            (x0, y0), (x1, y1) = poly[i], poly[(i + 1) % n]
            if y0 == y1:
                continue
            yb = min(y0, y1)                  # band [yb, yb + 1]
            py = yb + oy
            xc = x0 + (py - y0) * (x1 - x0) / (y1 - y0)
            # points with x + ox < xc see the crossing
            k = int(np.ceil(xc - ox))         # x < k
            k = min(max(k, 0), W)
            cnt[yb, 0] += 1 if y1 > y0 else -1
            cnt[yb, k] -= 1 if y1 > y0 else -1
        out.append(np.cumsum(cnt, axis=1)[:, :W])
    return out


def region_from_boundary(lattice: str, steps):
    """Cells enclosed by a closed lattice path (Sec. 1.1: a domain is a union
    of faces), by the winding number of the path around each cell centre.

    Domino: returns (face [H-1, W-1] bool, W, H).  Lozenge: returns
    (up [H, W], dn [H, W], W, H); up(x,y) has corners (x,y), (x+1,y),
    (x+1,y+1) and dn(x,y) has (x,y), (x+1,y+1), (x,y+1).  The path is shifted
    so that its smallest coordinates are 0.
    """
    pts = [(0, 0)]
    for s in steps:
        dx, dy = _STEPS[lattice][s]
        pts.append((pts[-1][0] + dx, pts[-1][1] + dy))
    assert pts[-1] == (0, 0), "path not closed"
    assert len(set(pts[:-1])) == len(pts) - 1, "path not simple"
    x0, y0 = min(p[0] for p in pts), min(p[1] for p in pts)
    poly = [(x - x0, y - y0) for x, y in pts[:-1]]
    W = max(p[0] for p in poly) + 1
    H = max(p[1] for p in poly) + 1
    if lattice == DOMINO:
        (w,) = _crossings(poly, W, H, [(0.5, 0.5)])
        return (w[:H - 1, :W - 1] != 0), W, H
    wu, wd = _crossings(poly, W, H, [(2 / 3, 1 / 3), (1 / 3, 2 / 3)])
    up, dn = wu != 0, wd != 0
    up[H - 1, :] = False
    up[:, W - 1] = False
    dn[H - 1, :] = False
    dn[:, W - 1] = False
    return up, dn, W, H


def tiling_by_search(lattice: str, region):
    """Some tiling of a region by depth-first search (first uncovered cell
    in (y, x) order, every way of covering it); None if there is none."""
    if lattice == DOMINO:
        face, W, H = region
        cells = [(y, x) for y in range(H - 1) for x in range(W - 1) if face[y, x]]
        inside = set(cells)

        def partners(c):
            y, x = c
            return [(y, x + 1), (y + 1, x), (y, x - 1), (y - 1, x)]
    else:
        up, dn, W, H = region
        cells = [(y, x, t) for y in range(H) for x in range(W) for t in (0, 1)
                 if (up if t == 0 else dn)[y, x]]
        inside = set(cells)

        def partners(c):
            y, x, t = c
            # up(x,y) meets dn(x,y-1) across E1(x,y), dn(x,y) across E3(x,y)
            # and dn(x+1,y) across E2(x+1,y)
            if t == 0:
                return [(y - 1, x, 1), (y, x, 1), (y, x + 1, 1)]
            return [(y + 1, x, 0), (y, x, 0), (y, x - 1, 0)]
    order = sorted(cells)
    nbr = {c: [q for q in partners(c) if q in inside] for c in cells}
    free = {c: len(nbr[c]) for c in cells}      # uncovered partners of each cell
    covered = set()
    pairs = []

    def place(c, q, cand):
        covered.update((c, q))
        pairs.append((c, q))
        for r in nbr[c] + nbr[q]:
            if r not in covered:
                free[r] -= 1
                if free[r] <= 1:
                    cand.append(r)

    def unplace():
        c, q = pairs[-1]
        for r in nbr[c] + nbr[q]:
            if r not in covered:
                free[r] += 1
        pairs.pop()
        covered.difference_update((c, q))

    def propagate(cand):
        # cover every cell that has a single uncovered partner left; False on
        # a cell with none.  Returns (ok, number of dominoes placed).
        n = 0
        while cand:
            r = cand.pop()
            if r in covered:
                continue
            if free[r] == 0:
                return False, n
            if free[r] == 1:
                q = next(q for q in nbr[r] if q not in covered)
                place(r, q, cand)
                n += 1
        return True, n

    def solve(i):
        # the first uncovered cell is at or after position i
        while i < len(order) and order[i] in covered:
            i += 1
        if i == len(order):
            return True
        c = order[i]
        for q in nbr[c]:
            if q in covered:
                continue
            cand = []
            place(c, q, cand)
            ok, n = propagate(cand)
            if ok and solve(i + 1):
                return True
            for _ in range(n + 1):
                unplace()
        return False

    import sys
    sys.setrecursionlimit(max(10000, 4 * len(cells)))
    cand = [c for c in cells if free[c] <= 1]
    ok, _ = propagate(cand)
    if not ok or not solve(0):
        return None
    if lattice == DOMINO:
        st = np.zeros((2, H, W), dtype=np.uint8)
        for (y, x), (y2, x2) in pairs:
            if y2 == y:      # horizontal domino crosses the vertical edge between its squares
                st[1, y, max(x, x2)] = 1
            else:            # vertical domino crosses the horizontal edge between its squares
                st[0, max(y, y2), x] = 1
        return st
    st = np.zeros((3, H, W), dtype=np.uint8)
    for a, b in pairs:
        (y, x, t), (y2, x2, t2) = (a, b) if a[2] == 0 else (b, a)   # (up, down)
        if y2 == y - 1:
            st[0, y, x] = 1          # E1(x,y)
        elif x2 == x:
            st[2, y, x] = 1          # E3(x,y)
        else:
            st[1, y, x + 1] = 1      # E2(x+1,y)
    return st


def extreme(lattice: str, st: np.ndarray, top: bool) -> np.ndarray:
    """T_max (top) or T_min of the region tiled by `st` (Sec. 1.1): apply
    whole-class rotations while they move the height function pointwise up
    (down) until none does.  A class move with all decisions equal moves
    every rotated site of the class the same way."""
    st = st.copy()
    h, bad = height(lattice, st)
    assert bad == 0
    while True:
        moved = False
        for p in range(PASSES[lattice]):
            for up in (1, 0):
                trial = st.copy()
                apply_pass(lattice, trial, p, np.full(st.shape[1:], up, np.uint8))
                if np.array_equal(trial, st):
                    continue
                h2, _ = height(lattice, trial)
                better = np.all(h2 >= h) if top else np.all(h2 <= h)
                if better:
                    st, h, moved = trial, h2, True
        if not moved:
            return st


def cftp(lattice: str, st_top: np.ndarray, st_bot: np.ndarray, *, seed: int, stream: int = 0,
         t0: int = 64, tmax: int = 1 << 31, **thr):
    """Coupling from the past (Sec. 1.1.4): chains from T_max and T_min run the
    sweeps of negative times -T..-1 (absolute sweep indices 2^32 - T ..
    2^32 - 1), T doubling until they agree; returns (sample, T)."""
    T = t0
    while True:
        a, b = st_top.copy(), st_bot.copy()
        sweeps(lattice, a, seed=seed, stream=stream, sweep0=(1 << 32) - T, k=T, **thr)
        sweeps(lattice, b, seed=seed, stream=stream, sweep0=(1 << 32) - T, k=T, **thr)
        if np.array_equal(a, b):
            return a, T
        if 2 * T > tmax:
            raise RuntimeError("no coalescence within %d sweeps" % T)
        T *= 2


# --------------------------------------------------------------------------
# Domino shuffling: exact uniform sampling of the Aztec diamond (Sec. 3,
# shuffling algorithms; Elkies, Kuperberg, Larsen and Propp)
# --------------------------------------------------------------------------
def shuffle_bit(seed: int, stream: int, order: int, x: int, y: int, n: int) -> int:
    """Orientation draw of the 2x2 block created with lower-left cell (x, y)
    (cell coordinates centred on the diamond) when growing to order `order`
    in a run of final order n: 1 = two horizontal dominoes.  Word 0 of
    Philox4x32-10 with key = seed and counter ((y+n) << 16 | (x+n), order,
    0xFFFE0000, stream), compared with 2^31."""
    w = philox4x32_10([((y + n) << 16) | (x + n), order, 0xFFFE0000, stream],
                      [seed & 0xFFFFFFFF, seed >> 32])
    return 1 if int(w[0]) < (1 << 31) else 0


def aztec_shuffle(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """Uniform random tiling of the Aztec diamond of order n by domino
    shuffling, in the canonical layout of aztec(n).

    Cells are unit squares with lower-left corner (x, y), the diamond of order
    k being |x + 1/2| + |y + 1/2| <= k.  In order k a horizontal domino with
    left cell (x, y) goes north if x + y + k is even and south otherwise; a
    vertical one with bottom cell (x, y) goes east if x + y + k is even and
    west otherwise (the top row's domino goes north, the left column's
    west).  One step k -> k+1: delete the bad blocks (a north-going domino
    directly below a south-going one, an east-going one directly left of a
    west-going one: they would pass through each other), move every other
    domino one cell in its direction, and fill the cells of order k+1 left
    empty, which form disjoint 2x2 blocks, block by block, taking the lowest
    then leftmost empty cell as a block's lower-left corner: two horizontal
    dominoes if the block's draw says so, else two vertical ones."""
    doms = {}                      # (x, y) of the left / bottom cell -> 0 horizontal, 1 vertical
    for k in range(n):
        def goes(x, y, o):
            even = (x + y + k) % 2 == 0
            if o == 0:
                return (0, 1) if even else (0, -1)
            return (1, 0) if even else (-1, 0)
        bad = set()
        for (x, y), o in doms.items():
            if o == 0 and (x + y + k) % 2 == 0 and doms.get((x, y + 1)) == 0:
                bad.update(((x, y), (x, y + 1)))
            if o == 1 and (x + y + k) % 2 == 0 and doms.get((x + 1, y)) == 1:
                bad.update(((x, y), (x + 1, y)))
        moved = {}
        for (x, y), o in doms.items():
            if (x, y) in bad:
                continue
            dx, dy = goes(x, y, o)
            moved[(x + dx, y + dy)] = o
        K = k + 1
        covered = set()
        for (x, y), o in moved.items():
            for c in (((x, y), (x + 1, y)) if o == 0 else ((x, y), (x, y + 1))):
                assert c not in covered
                covered.add(c)
        empty = sorted(((x, y) for y in range(-K, K) for x in range(-K, K)
                        if abs(x + 0.5) + abs(y + 0.5) <= K and (x, y) not in covered),
                       key=lambda c: (c[1], c[0]))
        filled = set()
        for (x, y) in empty:
            if (x, y) in filled:
                continue
            block = ((x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1))
            assert all(c not in covered and c not in filled for c in block)
            filled.update(block)
            if shuffle_bit(seed, stream, K, x, y, n):
                moved[(x, y)] = 0
                moved[(x, y + 1)] = 0
            else:
                moved[(x, y)] = 1
                moved[(x + 1, y)] = 1
        doms = moved
    W = 2 * n + 1
    st = np.zeros((2, W, W), dtype=np.uint8)
    for (x, y), o in doms.items():
        if o == 0:        # horizontal: crosses the vertical edge between its cells
            st[1, y + n, x + 1 + n] = 1
        else:             # vertical: crosses the horizontal edge between its cells
            st[0, y + 1 + n, x + n] = 1
    return st
