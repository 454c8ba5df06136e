"""Pins of the CPU oracle to what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a printed value
from the paper (Fig. 4, Fig. 5B/6), a published known-answer vector, a closed
form (Aztec 2^{n(n+1)/2}, Kasteleyn's product and determinant, MacMahon and
its q-analogue, alternating-sign-matrix counts and their 2-enumeration), an
exact stationarity identity of the transition matrix, or a statistical test
of the random chain against the exact Gibbs law.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle as O
from tests._enum import enumerate_states, pass_matrix, thresh_prob

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------------------
# Random numbers and hash
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    for row in _rows("philox_kat.txt"):
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_splitmix_known_answer_and_hash_properties():
    for row in _rows("splitmix64_kat.txt"):
        assert O.splitmix64(int(row[0], 16)) == int(row[1], 16)
    st = np.zeros((2, 5, 7), dtype=np.uint8)
    assert O.state_hash(st) == 0
    st.flat[13] = 1
    assert O.state_hash(st) == O.splitmix64(13)
    a = (np.random.default_rng(1).random(st.shape) < 0.5).astype(np.uint8)
    b = 1 - a
    full = np.ones_like(a)
    assert (O.state_hash(a) + O.state_hash(b)) % (1 << 64) == O.state_hash(full)


def test_site_uniform_is_uniform_and_planes_independent():
    # The bit-plane keyed u_v must be a uniform 32-bit number: P(u < t) = t/2^32.
    us = np.array([O.site_u(99, 3, 5, 1, r) for r in range(20000)], dtype=np.uint64)
    for t in (1 << 31, 1 << 30, 3 << 30, 123456789):
        frac = float(np.mean(us < t))
        p = t / 2.0 ** 32
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / us.size)
    bits = ((us[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    assert np.all(np.abs(bits.mean(0) - 0.5) < 0.02)
    c = np.corrcoef(bits.T)
    assert np.max(np.abs(c - np.eye(32))) < 0.05
    # neighbouring ranks, sweeps, passes and streams give different numbers
    assert O.site_u(99, 3, 5, 1, 7) != O.site_u(99, 3, 6, 1, 7)
    assert O.site_u(99, 3, 5, 1, 7) != O.site_u(99, 3, 5, 0, 7)
    assert O.site_u(99, 3, 5, 1, 7) != O.site_u(99, 4, 5, 1, 7)


# ---------------------------------------------------------------------------
# Worked examples printed in the paper
# ---------------------------------------------------------------------------
def _fig4_canonical():
    """Fig. 4 under the reading where East points to decreasing column."""
    m = np.array([[int(v) for v in r] for r in _rows("fig4_tilestate.txt")])
    H, W = m.shape
    st = np.zeros((2, H, W), dtype=np.uint8)
    for r in range(H):
        for c in range(W):
            s = m[r, c]
            x, y = W - 1 - c, H - 1 - r
            if s & 1: st[1, y, x] = 1          # N: edge (x,y)-(x,y+1)
            if s & 2: st[1, y - 1, x] = 1      # S: edge (x,y-1)-(x,y)
            if s & 4: st[0, y, x] = 1          # E: edge (x,y)-(x+1,y)
            if s & 8: st[0, y, x - 1] = 1      # W: edge (x-1,y)-(x,y)
    return m, st


def _tilestate(st):
    _, H, W = st.shape
    m = np.zeros((H, W), dtype=int)
    for y in range(H):
        for x in range(W):
            s = st[1, y, x] * 1 + (st[1, y - 1, x] * 2 if y > 0 else 0)
            s += st[0, y, x] * 4 + (st[0, y, x - 1] * 8 if x > 0 else 0)
            m[H - 1 - y, W - 1 - x] = s
    return m


def test_fig4_tilestate_round_trip_and_rotation():
    m, st = _fig4_canonical()
    # every edge is reported identically by both of its endpoints
    assert np.array_equal(_tilestate(st), m)
    # it is a domino tiling of the 4x4 square (all 16 faces covered once)
    assert O.domino_check(st, np.ones((4, 4), dtype=np.uint8)) == 0
    assert int(st.sum()) == 8
    # the centre vertex has tilestate 12 and is the only rotatable site
    codes = O.site_states(O.DOMINO, st, 0) + O.site_states(O.DOMINO, st, 1)
    assert codes[2, 2] == 2 and int((codes > 0).sum()) == 1
    # rotating it down changes exactly five vertex states: 12 -> 3 at the
    # centre, and one bit at each of its four neighbours
    nxt = st.copy()
    O.apply_pass(O.DOMINO, nxt, 0, np.zeros((5, 5), dtype=np.uint8))
    m2 = _tilestate(nxt)
    assert int((m2 != m).sum()) == 5
    assert m2[2, 2] == 3
    assert O.domino_check(nxt, np.ones((4, 4), dtype=np.uint8)) == 0


def _fig6_config():
    lines = open(os.path.join(GOLDEN, "fig6_sixvertex.txt")).read().splitlines()
    lines = [ln for ln in lines if ln.strip() and not ln.startswith("#")]
    i_h = lines.index("[heights]")
    paths = [[tuple(float(v) for v in p.split(",")) for p in ln.split()]
             for ln in lines[1:i_h]]
    heights = np.array([[int(v) for v in ln.split()] for ln in lines[i_h + 1:]])
    # vertex (X, Y) of a 6-wide box (N = 6) from figure coordinates; the
    # figure's 4 rows sit at Y = 1..4 and paths leaving the top are continued
    # straight up through the two spare rows.
    N = 6
    st = np.zeros((2, N + 2, N + 2), dtype=np.uint8)

    def X(x): return int(round((x + 1.5) / 0.5)) + 1
    def Y(y): return int(round((y + 1.0) / 0.5)) + 1

    for path in paths:
        for (x0, y0), (x1, y1) in zip(path, path[1:]):
            if y0 == y1:                       # horizontal run
                lo, hi = sorted((X(x0), X(x1)))
                for xx in range(lo, hi):
                    st[0, Y(y0), xx] = 1
            else:                              # vertical run
                lo, hi = sorted((Y(y0), Y(y1)))
                for yy in range(lo, hi):
                    st[1, yy, X(x0)] = 1
        xe, ye = path[-1]
        if ye > 0.5:                           # left through the top: continue up
            for yy in range(Y(0.5), N + 1):
                st[1, yy, X(xe)] = 1
    return st, heights


def test_fig5b_ice_rule_and_fig6_heights():
    st, heights = _fig6_config()
    # the printed configuration obeys the ice rule at all 24 vertices
    for Y in range(1, 5):
        for X in range(1, 7):
            assert O.sixv_vertex_type(st, X, Y) >= 0
    h, bad = O.height(O.SIXV, st)
    assert bad == 0
    assert np.array_equal(h[0:5, 0:7], heights)


# ---------------------------------------------------------------------------
# Closed-form counts via brute-force enumeration under elementary moves
# ---------------------------------------------------------------------------
def kasteleyn_count(m, n):
    """Number of domino tilings of an m x n rectangle (Kasteleyn 1961)."""
    prod = 1.0
    for j in range(1, (m + 1) // 2 + 1):
        for k in range(1, (n + 1) // 2 + 1):
            prod *= 4 * math.cos(math.pi * j / (m + 1)) ** 2 + 4 * math.cos(math.pi * k / (n + 1)) ** 2
    return round(prod)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_aztec_count(n):
    states, _ = enumerate_states(O.DOMINO, O.aztec(n))
    assert len(states) == 2 ** (n * (n + 1) // 2)
    for st in states:
        assert O.domino_check(st, _aztec_faces(n)) == 0


def _aztec_faces(n):
    W = 2 * n
    fm = np.zeros((W, W), dtype=np.uint8)
    for y in range(W):
        for x in range(W):
            fm[y, x] = abs(x + 0.5 - n) + abs(y + 0.5 - n) <= n
    return fm


@pytest.mark.parametrize("w,h", [(2, 5), (4, 3), (4, 4), (5, 4), (6, 6)])
def test_rectangle_count(w, h):
    states, _ = enumerate_states(O.DOMINO, O.rect(w, h))
    assert len(states) == kasteleyn_count(w, h)
    for st in states[:: max(1, len(states) // 50)]:
        assert O.domino_check(st, np.ones((h, w), dtype=np.uint8)) == 0


def test_rectangle_untileable():
    with pytest.raises(ValueError):
        O.rect(3, 5)


def kasteleyn_det(w, h, weights):
    """|det K| with Kasteleyn weights (horizontal real, vertical times i)."""
    faces = [(x, y) for y in range(h) for x in range(w)]
    black = [f for f in faces if (f[0] + f[1]) % 2 == 0]
    white = [f for f in faces if (f[0] + f[1]) % 2 == 1]
    bi = {f: i for i, f in enumerate(black)}
    wi = {f: i for i, f in enumerate(white)}
    K = np.zeros((len(black), len(white)), dtype=complex)
    for (x, y) in black:
        # horizontal dual edges cross vertical primal edges Vt
        for dx in (-1, 1):
            nb = (x + dx, y)
            if nb in wi:
                K[bi[(x, y)], wi[nb]] = weights[1, y, max(x, x + dx)]
        # vertical dual edges cross horizontal primal edges Hz
        for dy in (-1, 1):
            nb = (x, y + dy)
            if nb in wi:
                K[bi[(x, y)], wi[nb]] = 1j * weights[0, max(y, y + dy), x]
    return abs(np.linalg.det(K))


def test_weighted_partition_function_matches_kasteleyn():
    w, h = 4, 4
    rng = np.random.default_rng(5)
    wts = np.exp(0.5 * rng.standard_normal((2, h + 1, w + 1)))
    states, _ = enumerate_states(O.DOMINO, O.rect(w, h))
    Z = sum(O.domino_weight(st, wts) for st in states)
    assert Z == pytest.approx(kasteleyn_det(w, h, wts), rel=1e-10)


def macmahon(a, b, c):
    num = den = 1
    for i in range(1, a + 1):
        for j in range(1, b + 1):
            for k in range(1, c + 1):
                num *= i + j + k - 1
                den *= i + j + k - 2
    return num // den


@pytest.mark.parametrize("a,b,c", [(1, 1, 1), (2, 2, 2), (1, 2, 3), (2, 3, 2), (3, 3, 3)])
def test_hexagon_count(a, b, c):
    states, _ = enumerate_states(O.LOZENGE, O.hexagon(a, b, c))
    assert len(states) == macmahon(a, b, c)
    st0 = states[0]
    for st in states[:: max(1, len(states) // 60)]:
        assert O.lozenge_check(st) == 0
        # the covered triangles are the same as for the starting tiling
        assert O.lozenge_check(st, *_tri_masks(st0)) == 0


def _tri_masks(st):
    _, H, W = st.shape
    up = np.zeros((H, W), dtype=np.uint8)
    dn = np.zeros((H, W), dtype=np.uint8)
    g = lambda k, x, y: st[k, y, x] if 0 <= x < W and 0 <= y < H else 0
    for y in range(H):
        for x in range(W):
            up[y, x] = g(0, x, y) + g(1, x + 1, y) + g(2, x, y)
            dn[y, x] = g(2, x, y) + g(1, x, y) + g(0, x, y + 1)
    return up, dn


def _poly_mul(p, q):
    r = [0] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            r[i + j] += a * b
    return r


def _poly_div_exact(p, q):
    p = list(p)
    out = [0] * (len(p) - len(q) + 1)
    for i in range(len(out)):
        c = p[i] // q[0]
        out[i] = c
        for j, b in enumerate(q):
            p[i + j] -= c * b
    assert all(v == 0 for v in p)
    return out


def q_macmahon(a, b, c):
    """Coefficients of prod (1 - q^{i+j+k-1}) / (1 - q^{i+j+k-2})."""
    num, den = [1], [1]
    for i in range(1, a + 1):
        for j in range(1, b + 1):
            for k in range(1, c + 1):
                e1, e2 = i + j + k - 1, i + j + k - 2
                num = _poly_mul(num, [1] + [0] * (e1 - 1) + [-1])
                den = _poly_mul(den, [1] + [0] * (e2 - 1) + [-1])
    return _poly_div_exact(num, den)


def _volume(st, h0):
    h, bad = O.height(O.LOZENGE, st)
    assert bad == 0
    m = h0 != O.HEIGHT_NONE
    return int((h[m] - h0[m]).sum())


@pytest.mark.parametrize("a,b,c", [(2, 2, 2), (2, 3, 2)])
def test_hexagon_volume_generating_function(a, b, c):
    st0 = O.hexagon(a, b, c)
    h0, bad = O.height(O.LOZENGE, st0)
    assert bad == 0
    states, _ = enumerate_states(O.LOZENGE, st0)
    vols = [_volume(st, h0) for st in states]
    assert min(vols) == 0
    hist = np.bincount(vols)
    want = q_macmahon(a, b, c)
    assert list(hist) == want[: len(hist)] and sum(want) == len(states)


ASM = {1: 1, 2: 2, 3: 7, 4: 42, 5: 429}


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_dwbc_counts_are_asm_numbers(N):
    states, _ = enumerate_states(O.SIXV, O.dwbc(N))
    assert len(states) == ASM[N]
    for st in states:
        assert O.sixv_check_dwbc(st) == 0


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_dwbc_two_enumeration(N):
    # a = b = 1, c = sqrt(2): Z = 2^{N/2} * 2^{N(N-1)/2} (the 2-enumeration of ASMs)
    w6 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]
    states, _ = enumerate_states(O.SIXV, O.dwbc(N))
    Z = sum(O.sixv_weight(st, w6) for st in states)
    assert Z == pytest.approx(2 ** (N / 2) * 2 ** (N * (N - 1) / 2), rel=1e-12)


# ---------------------------------------------------------------------------
# Exact stationarity of every heat-bath pass (no randomness involved)
# ---------------------------------------------------------------------------
def _check_stationary(lattice, states, index, weights, prob_up, tol):
    pi = np.array(weights, dtype=np.float64)
    pi /= pi.sum()
    for p in range(O.PASSES[lattice]):
        P = pass_matrix(lattice, states, index, p, prob_up)
        assert np.allclose(P.sum(1), 1.0, atol=1e-12)
        assert np.max(np.abs(pi @ P - pi)) <= tol


def test_stationary_domino_uniform():
    states, index = enumerate_states(O.DOMINO, O.aztec(3))
    _check_stationary(O.DOMINO, states, index, [1.0] * len(states),
                      lambda st, y, x: thresh_prob(1 << 31), 1e-15)


@pytest.mark.parametrize("shape", ["aztec3", "rect4x4"])
def test_stationary_domino_weighted(shape):
    st0 = O.aztec(3) if shape == "aztec3" else O.rect(4, 4)
    rng = np.random.default_rng(11)
    wts = np.exp(0.5 * rng.standard_normal(st0.shape))
    t = O.domino_thresholds(wts)
    states, index = enumerate_states(O.DOMINO, st0)
    # thresholds are floor(2^32 p): each probability is within 2^-32 of exact
    _check_stationary(O.DOMINO, states, index, [O.domino_weight(s, wts) for s in states],
                      lambda st, y, x: thresh_prob(t[y, x]), 1e-8)


def test_stationary_lozenge_q():
    q = 0.7
    st0 = O.hexagon(2, 2, 2)
    h0, _ = O.height(O.LOZENGE, st0)
    ta, tr = O.lozenge_thresholds(q)
    assert ta + tr == 1 << 32
    states, index = enumerate_states(O.LOZENGE, st0)
    _check_stationary(O.LOZENGE, states, index, [q ** _volume(s, h0) for s in states],
                      lambda st, y, x: thresh_prob(ta), 1e-8)


def _sixv_index(st, X, Y):
    return (int(st[1, Y + 1, X]) | (int(st[0, Y + 1, X + 1]) << 1) |
            (int(st[0, Y, X + 1]) << 2) | (int(st[0, Y, X - 1]) << 3))


@pytest.mark.parametrize("w6", [[1, 1, 1, 1, math.sqrt(2), math.sqrt(2)],
                                [0.7, 1.3, 0.4, 1.9, 1.1, 0.6]])
def test_stationary_sixv(w6):
    t16 = O.sixv_thresholds(w6)
    states, index = enumerate_states(O.SIXV, O.dwbc(4))
    _check_stationary(O.SIXV, states, index, [O.sixv_weight(s, w6) for s in states],
                      lambda st, Y, X: thresh_prob(t16[_sixv_index(st, X, Y)]), 1e-8)


def test_sixv_two_colour_parallel_pass_is_not_stationary():
    # Faces of one checkerboard colour share corner vertices; updating them
    # together (classes (0,0) and (1,1) at once) breaks the Gibbs law at
    # c = sqrt(2), which is why a sweep uses the four parity classes.
    w6 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]
    t16 = O.sixv_thresholds(w6)
    states, index = enumerate_states(O.SIXV, O.dwbc(4))
    pi = np.array([O.sixv_weight(s, w6) for s in states])
    pi /= pi.sum()
    n = len(states)
    P = np.zeros((n, n))
    import itertools
    for a, st in enumerate(states):
        sites = []
        for p in (0, 1):
            codes = O.site_states(O.SIXV, st, p)
            for Y, X in zip(*np.nonzero(codes)):
                sites.append((p, Y, X, thresh_prob(t16[_sixv_index(st, X, Y)])))
        for choice in itertools.product((0, 1), repeat=len(sites)):
            pr = 1.0
            decs = [np.zeros(st.shape[1:], dtype=np.uint8) for _ in range(2)]
            for (p, Y, X, q), c in zip(sites, choice):
                decs[p][Y, X] = c
                pr *= q if c else 1 - q
            nxt = st.copy()
            O.apply_pass(O.SIXV, nxt, 0, decs[0])
            O.apply_pass(O.SIXV, nxt, 1, decs[1])
            P[a, index[nxt.tobytes()]] += pr
    assert np.max(np.abs(pi @ P - pi)) > 1e-3


# ---------------------------------------------------------------------------
# Thresholds against the global definition of the Gibbs weight
# ---------------------------------------------------------------------------
def test_domino_threshold_is_local_conditional_probability():
    st0 = O.aztec(3)
    rng = np.random.default_rng(2)
    wts = np.exp(0.5 * rng.standard_normal(st0.shape))
    t = O.domino_thresholds(wts)
    states, _ = enumerate_states(O.DOMINO, st0)
    checked = 0
    for st in states[:40]:
        for p in (0, 1):
            codes = O.site_states(O.DOMINO, st, p)
            for y, x in zip(*np.nonzero(codes)):
                up, dn = st.copy(), st.copy()
                d = np.zeros(codes.shape, dtype=np.uint8)
                d[y, x] = 1
                base = (codes == 2).astype(np.uint8)
                O.apply_pass(O.DOMINO, up, p, np.maximum(base, d))
                O.apply_pass(O.DOMINO, dn, p, base * (1 - d))
                wu, wd = O.domino_weight(up, wts), O.domino_weight(dn, wts)
                assert abs(thresh_prob(t[y, x]) - wu / (wu + wd)) <= 2.0 ** -32
                checked += 1
    assert checked > 50
    assert np.all(O.domino_thresholds(np.ones(st0.shape)) == 1 << 31)


def test_sixv_table_is_local_conditional_probability():
    w6 = [0.7, 1.3, 0.4, 1.9, 1.1, 0.6]
    t16 = O.sixv_thresholds(w6)
    states, _ = enumerate_states(O.SIXV, O.dwbc(5))
    seen = set()
    for st in states:
        for p in range(4):
            codes = O.site_states(O.SIXV, st, p)
            for Y, X in zip(*np.nonzero(codes)):
                base = (codes == 2).astype(np.uint8)
                d = np.zeros(codes.shape, dtype=np.uint8)
                d[Y, X] = 1
                up, dn = st.copy(), st.copy()
                O.apply_pass(O.SIXV, up, p, np.maximum(base, d))
                O.apply_pass(O.SIXV, dn, p, base * (1 - d))
                wu, wd = O.sixv_weight(up, w6), O.sixv_weight(dn, w6)
                idx = _sixv_index(st, X, Y)
                assert abs(thresh_prob(t16[idx]) - wu / (wu + wd)) <= 2.0 ** -32
                seen.add(idx)
    assert len(seen) >= 10
    # a = b = 1, c = sqrt(2): P(UP) = 1 / (1 + 2^{2-k}), k = c-corners after the flip
    t = O.sixv_thresholds([1, 1, 1, 1, math.sqrt(2), math.sqrt(2)])
    allowed = {math.floor(2 ** 32 / (1 + 2.0 ** (2 - k))) for k in range(5)}
    assert set(int(v) for v in t) <= allowed


# ---------------------------------------------------------------------------
# The random chain samples the Gibbs law (chi-square on tiny domains)
# ---------------------------------------------------------------------------
def _chi2_pvalue(counts, probs):
    from scipy.stats import chisquare
    n = counts.sum()
    return chisquare(counts, probs * n).pvalue


@pytest.mark.parametrize("case", ["aztec3", "hex222", "dwbc4"])
def test_random_chain_chi_square(case):
    if case == "aztec3":
        lat, st0, kw = O.DOMINO, O.aztec(3), dict(t_scalar=1 << 31)
        states, index = enumerate_states(lat, st0)
        pi = np.ones(len(states))
    elif case == "hex222":
        lat, st0 = O.LOZENGE, O.hexagon(2, 2, 2)
        ta, _ = O.lozenge_thresholds(1.5)
        kw = dict(t_scalar=ta)
        h0, _ = O.height(O.LOZENGE, st0)
        states, index = enumerate_states(lat, st0)
        pi = np.array([1.5 ** _volume(s, h0) for s in states])
    else:
        lat, st0 = O.SIXV, O.dwbc(4)
        w6 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]
        kw = dict(t16=O.sixv_thresholds(w6))
        states, index = enumerate_states(lat, st0)
        pi = np.array([O.sixv_weight(s, w6) for s in states])
    pi = pi / pi.sum()
    counts = np.zeros(len(states))
    st = st0.copy()
    O.sweeps(lat, st, seed=2024, stream=1, sweep0=0, k=30, **kw)
    thin, nsamp = 6, 3000
    for i in range(nsamp):
        O.sweeps(lat, st, seed=2024, stream=1, sweep0=30 + i * thin, k=thin, **kw)
        counts[index[st.tobytes()]] += 1
    assert _chi2_pvalue(counts, pi) > 1e-4


# ---------------------------------------------------------------------------
# Height-function invariants under the chain
# ---------------------------------------------------------------------------
def test_domino_height_invariants():
    n = 6
    st0 = O.aztec(n)
    h0, bad = O.height(O.DOMINO, st0)
    assert bad == 0
    st = st0.copy()
    O.sweeps(O.DOMINO, st, seed=3, k=40, t_scalar=1 << 31)
    h, bad = O.height(O.DOMINO, st)
    assert bad == 0
    dom = h0 != O.HEIGHT_NONE
    assert np.array_equal(h != O.HEIGHT_NONE, dom)
    # heights mod 4 are fixed by position; boundary heights are fixed
    assert np.all(((h - h0) % 4)[dom] == 0)
    fm = _aztec_faces(n)
    W = 2 * n + 1
    for y in range(W):
        for x in range(W):
            if not dom[y, x]:
                continue
            around = [fm[yy, xx] if 0 <= xx < 2 * n and 0 <= yy < 2 * n else 0
                      for xx, yy in ((x, y), (x - 1, y), (x, y - 1), (x - 1, y - 1))]
            if not all(around):
                assert h[y, x] == h0[y, x]
    # |dh| = 1 on uncrossed and 3 on crossed domain edges
    for y in range(W):
        for x in range(W - 1):
            if dom[y, x] and dom[y, x + 1]:
                assert abs(int(h[y, x + 1]) - int(h[y, x])) == (3 if st[0, y, x] else 1)
    # an elementary rotation changes the height at its site by 4 and nowhere else
    codes = O.site_states(O.DOMINO, st, 0)
    y, x = [int(v[0]) for v in np.nonzero(codes)]
    nxt = st.copy()
    dec = (codes == 2).astype(np.uint8)
    dec[y, x] ^= 1
    O.apply_pass(O.DOMINO, nxt, 0, dec)
    h2, _ = O.height(O.DOMINO, nxt)
    diff = (h2 - h)[dom]
    assert int((diff != 0).sum()) == 1 and abs(int(diff[diff != 0][0])) == 4


def test_lozenge_rotation_changes_height_by_one():
    st = O.hexagon(3, 4, 2)
    O.sweeps(O.LOZENGE, st, seed=9, k=20, t_scalar=1 << 31)
    h, bad = O.height(O.LOZENGE, st)
    assert bad == 0
    for p in range(3):
        codes = O.site_states(O.LOZENGE, st, p)
        for y, x in list(zip(*np.nonzero(codes)))[:3]:
            nxt = st.copy()
            dec = (codes == 2).astype(np.uint8)
            dec[y, x] ^= 1
            O.apply_pass(O.LOZENGE, nxt, p, dec)
            h2, _ = O.height(O.LOZENGE, nxt)
            d = h2.astype(np.int64) - h
            assert int((d != 0).sum()) == 1
            # going UP adds a cube
            assert int(d[y, x]) == (1 if codes[y, x] == 1 else -1)


def test_sixv_flip_raises_face_height_by_two():
    st = O.dwbc(6)
    O.sweeps(O.SIXV, st, seed=4, k=10, t16=O.sixv_thresholds([1, 1, 1, 1, 1, 1]))
    h, bad = O.height(O.SIXV, st)
    assert bad == 0
    codes = O.site_states(O.SIXV, st, 0)
    Y, X = [int(v[0]) for v in np.nonzero(codes)]
    nxt = st.copy()
    dec = (codes == 2).astype(np.uint8)
    dec[Y, X] ^= 1
    O.apply_pass(O.SIXV, nxt, 0, dec)
    h2, bad = O.height(O.SIXV, nxt)
    assert bad == 0
    d = h2 - h
    assert int((d != 0).sum()) == 1
    assert int(d[Y, X]) == (2 if codes[Y, X] == 1 else -2)
    # boundary heights of the domain-wall boundary are fixed
    N = 6
    ar = np.arange(N + 1)
    assert np.array_equal(h[0, :], ar)          # bottom externals occupied
    assert np.array_equal(h[:, 0], ar)          # left externals occupied
    assert np.array_equal(h[N, :], N - ar)      # top externals empty
    assert np.array_equal(h[:, N], N - ar)      # right externals empty


# ---------------------------------------------------------------------------
# Extreme tilings, regions from a boundary path, coupling from the past
# (Sec. 1.1 T_max / T_min and Thurston's algorithm; Sec. 1.1.4)
# ---------------------------------------------------------------------------
def _enum_case(case):
    if case == "aztec3":
        return O.DOMINO, O.aztec(3)
    if case == "rect4x3":
        return O.DOMINO, O.rect(4, 3)
    if case == "hex223":
        return O.LOZENGE, O.hexagon(2, 2, 3)
    return O.SIXV, O.dwbc(4)


@pytest.mark.parametrize("case", ["aztec3", "rect4x3", "hex223", "dwbc4"])
def test_extremes_bound_every_tiling(case):
    # T_max / T_min are the pointwise largest / smallest height functions
    # among all tilings of the domain (enumerated by elementary moves)
    lat, st0 = _enum_case(case)
    states, _ = enumerate_states(lat, st0)
    hs = np.stack([O.height(lat, s)[0] for s in states])
    hmax, hmin = hs.max(axis=0), hs.min(axis=0)
    top, bot = O.extreme(lat, st0, True), O.extreme(lat, st0, False)
    assert np.array_equal(O.height(lat, top)[0], hmax)
    assert np.array_equal(O.height(lat, bot)[0], hmin)


def _aztec_path(n):
    # boundary of the Aztec diamond of order n, counter-clockwise from the
    # lower end of its left column of faces: staircases of unit steps
    steps = []
    for _ in range(n):
        steps += [3, 0]          # down-right staircase (lower left edge)
    for _ in range(n):
        steps += [0, 1]          # up-right (lower right edge)
    for _ in range(n):
        steps += [1, 2]          # up-left (upper right edge)
    for _ in range(n):
        steps += [2, 3]          # down-left (upper left edge)
    return steps


DOMINO_SHAPES = {
    "square4": [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4,
    "L": [0] * 4 + [1] * 2 + [2] * 2 + [1] * 2 + [2] * 2 + [3] * 4,
    "U": [0] * 6 + [1] * 4 + [2] * 2 + [3] * 2 + [2] * 2 + [1] * 2 + [2] * 2 + [3] * 4,
    "aztec4": _aztec_path(4),
}


def test_region_cells_and_search_tilings():
    face, W, H = O.region_from_boundary(O.DOMINO, DOMINO_SHAPES["square4"])
    assert face.sum() == 16 and (W, H) == (5, 5)
    face, W, H = O.region_from_boundary(O.DOMINO, DOMINO_SHAPES["U"])
    assert face.sum() == 20
    assert not face[2, 2] and not face[3, 3] and face[1, 2]
    face, W, H = O.region_from_boundary(O.DOMINO, _aztec_path(4))
    assert np.array_equal(face, _aztec_faces(4))
    for name, steps in DOMINO_SHAPES.items():
        reg = O.region_from_boundary(O.DOMINO, steps)
        st = O.tiling_by_search(O.DOMINO, reg)
        assert st is not None and O.domino_check(st, reg[0]) == 0, name
    # hexagon with sides (a, b, c) along +x, +x+y, +y: 2(ab + bc + ca) triangles,
    # and its tilings by search count like MacMahon's box
    a, b, c = 2, 1, 2
    steps = [0] * a + [2] * b + [1] * c + [3] * a + [5] * b + [4] * c
    up, dn, W, H = O.region_from_boundary(O.LOZENGE, steps)
    assert up.sum() + dn.sum() == 2 * (a * b + b * c + c * a)
    st = O.tiling_by_search(O.LOZENGE, (up, dn, W, H))
    assert st is not None and O.lozenge_check(st, up, dn) == 0
    states, _ = enumerate_states(O.LOZENGE, st)
    # MacMahon: prod over the box of (i+j+k-1)/(i+j+k-2) = 2 * 3/2 * 3/2 * 4/3 = 6
    assert len(states) == 6


def test_search_finds_no_tiling_of_untileable_regions():
    # 4 x 4 square without two opposite corners (same colour): no tiling
    steps = [0] * 3 + [1] * 3 + [2] + [1] + [2] * 3 + [3] * 3 + [0] + [3]
    reg = O.region_from_boundary(O.DOMINO, steps)
    assert reg[0].sum() == 14
    assert O.tiling_by_search(O.DOMINO, reg) is None


@pytest.mark.parametrize("case", ["aztec2", "hex222", "dwbc3"])
def test_cftp_samples_exactly(case):
    # coupling from the past returns exact samples: chi-square of the outputs
    # over independent seeds against the Gibbs law
    if case == "aztec2":
        lat, st0, kw = O.DOMINO, O.aztec(2), dict(t_scalar=1 << 31)
        states, index = enumerate_states(lat, st0)
        pi = np.ones(len(states))
    elif case == "hex222":
        lat, st0 = O.LOZENGE, O.hexagon(2, 2, 2)
        ta, _ = O.lozenge_thresholds(1.5)
        kw = dict(t_scalar=ta)
        h0, _ = O.height(O.LOZENGE, st0)
        states, index = enumerate_states(lat, st0)
        pi = np.array([1.5 ** _volume(s, h0) for s in states])
    else:
        lat, st0 = O.SIXV, O.dwbc(3)
        w6 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]
        kw = dict(t16=O.sixv_thresholds(w6))
        states, index = enumerate_states(lat, st0)
        pi = np.array([O.sixv_weight(s, w6) for s in states])
    pi = pi / pi.sum()
    top, bot = O.extreme(lat, st0, True), O.extreme(lat, st0, False)
    counts = np.zeros(len(states))
    for seed in range(600):
        s, T = O.cftp(lat, top, bot, seed=seed, stream=7, t0=2, **kw)
        counts[index[s.tobytes()]] += 1
    assert _chi2_pvalue(counts, pi) > 1e-4


def test_coupled_chains_stay_ordered():
    # the heat-bath move with shared random numbers is monotone: the chain
    # from T_max stays pointwise above the chain from T_min at every sweep
    for lat, st0, kw in ((O.DOMINO, O.aztec(5), dict(t_scalar=0x70000000)),
                         (O.LOZENGE, O.hexagon(3, 4, 2), dict(t_scalar=0x9000_0000)),
                         (O.SIXV, O.dwbc(6), dict(t16=O.sixv_thresholds([1, 1, 1, 1, 1.7, 1.7])))):
        a, b = O.extreme(lat, st0, True), O.extreme(lat, st0, False)
        for s in range(40):
            O.sweeps(lat, a, seed=9, sweep0=s, k=1, **kw)
            O.sweeps(lat, b, seed=9, sweep0=s, k=1, **kw)
            assert np.all(O.height(lat, a)[0] >= O.height(lat, b)[0]), (lat, s)


# ---------------------------------------------------------------------------
# Volume weights (Sec. 1.1.1): W(T) = prod_v q_v^h(v)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["aztec3", "rect4x3", "hex222"])
def test_volume_thresholds_are_stationary(case):
    lat, st0 = {"aztec3": (O.DOMINO, O.aztec(3)), "rect4x3": (O.DOMINO, O.rect(4, 3)),
                "hex222": (O.LOZENGE, O.hexagon(2, 2, 2))}[case]
    rng = np.random.default_rng(5)
    q = np.exp(0.4 * rng.standard_normal(st0.shape[1:]))
    t = O.volume_thresholds(lat, q)
    states, index = enumerate_states(lat, st0)
    _check_stationary(lat, states, index, [O.volume_weight(lat, s, q) for s in states],
                      lambda st, y, x: thresh_prob(t[y, x]), 1e-8)


def test_volume_weight_one_is_uniform_and_rotation_moves_height_by_four():
    st = O.aztec(6)
    t = O.volume_thresholds(O.DOMINO, np.ones(st.shape[1:]))
    assert np.all(t == 1 << 31)
    O.sweeps(O.DOMINO, st, seed=8, k=30, t_scalar=1 << 31)
    # the parity rule: UP raises h(v) by 4 at x + y even and lowers it at odd
    h0, _ = O.height(O.DOMINO, st)
    for p in range(2):
        codes = O.site_states(O.DOMINO, st, p)
        ys, xs = np.nonzero(codes == 1)          # DOWN sites of this class
        y, x = ys[0], xs[0]
        dec = (codes == 2).astype(np.uint8)
        dec[y, x] = 1
        nxt = st.copy()
        O.apply_pass(O.DOMINO, nxt, p, dec)
        h1, _ = O.height(O.DOMINO, nxt)
        diff = h1 - h0
        assert diff[y, x] == (4 if (x + y) % 2 == 0 else -4)
        diff[y, x] = 0
        assert not np.any(diff[h0 != O.HEIGHT_NONE])


# ---------------------------------------------------------------------------
# Random pass order (the RandomWalk of Sec. 2.2 picks each step's colour at
# random)
# ---------------------------------------------------------------------------
def test_slot_colours_uniform_and_from_philox():
    from scipy.stats import chisquare
    for P in (2, 3, 4):
        cols = np.array([O.slot_colour(99, 5, s, i, P) for s in range(3000) for i in range(P)])
        assert cols.min() >= 0 and cols.max() < P
        assert chisquare(np.bincount(cols, minlength=P)).pvalue > 1e-4
        # pairs of consecutive slots are independent
        pairs = cols[:-1] * P + cols[1:]
        assert chisquare(np.bincount(pairs, minlength=P * P)).pvalue > 1e-4
    # the draw is word 0 of the Random123 Philox output for its counter, scaled
    out = O.philox4x32_10([0xFFFFFFFF, 17, 0xFFFF0002, 5], [99, 0])
    assert O.slot_colour(99, 5, 17, 2, 3) == (int(out[0]) * 3) >> 32


@pytest.mark.parametrize("case", ["aztec3", "hex222", "dwbc4"])
def test_random_order_chain_chi_square(case):
    if case == "aztec3":
        lat, st0, kw = O.DOMINO, O.aztec(3), dict(t_scalar=1 << 31)
        states, index = enumerate_states(lat, st0)
        pi = np.ones(len(states))
    elif case == "hex222":
        lat, st0 = O.LOZENGE, O.hexagon(2, 2, 2)
        ta, _ = O.lozenge_thresholds(1.5)
        kw = dict(t_scalar=ta)
        h0, _ = O.height(O.LOZENGE, st0)
        states, index = enumerate_states(lat, st0)
        pi = np.array([1.5 ** _volume(s, h0) for s in states])
    else:
        lat, st0 = O.SIXV, O.dwbc(4)
        w6 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]
        kw = dict(t16=O.sixv_thresholds(w6))
        states, index = enumerate_states(lat, st0)
        pi = np.array([O.sixv_weight(s, w6) for s in states])
    pi = pi / pi.sum()
    counts = np.zeros(len(states))
    st = st0.copy()
    O.sweeps(lat, st, seed=7, stream=2, sweep0=0, k=30, random_order=True, **kw)
    for i in range(3000):
        O.sweeps(lat, st, seed=7, stream=2, sweep0=30 + 6 * i, k=6, random_order=True, **kw)
        counts[index[st.tobytes()]] += 1
    assert _chi2_pvalue(counts, pi) > 1e-4
    # and the order really differs from the fixed one
    a, b = st0.copy(), st0.copy()
    O.sweeps(lat, a, seed=7, k=5, **kw)
    O.sweeps(lat, b, seed=7, k=5, random_order=True, **kw)
    assert not np.array_equal(a, b)


# ---------------------------------------------------------------------------
# Domino shuffling (Sec. 3): exact uniform tilings of the Aztec diamond
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 5, 13, 30])
def test_shuffling_gives_tilings_of_the_diamond(n):
    for seed in range(3):
        st = O.aztec_shuffle(n, seed, stream=seed)
        assert O.domino_check(st, _aztec_faces(n)) == 0
        assert O.height(O.DOMINO, st)[1] == 0


def test_shuffling_is_uniform():
    # every one of the 2^(n(n+1)/2) = 64 tilings of order 3 equally likely
    states, index = enumerate_states(O.DOMINO, O.aztec(3))
    assert len(states) == 64
    counts = np.zeros(64)
    for seed in range(6400):
        counts[index[O.aztec_shuffle(3, seed).tobytes()]] += 1
    assert _chi2_pvalue(counts, np.full(64, 1 / 64)) > 1e-4


# ---------------------------------------------------------------------------
# North / south / east / west domino types (Sec. 4's arctic-circle pictures)
# ---------------------------------------------------------------------------
def _nsew_types(counts):
    """Face type 0..3 where exactly one counter is set, -1 where none."""
    tot = counts.sum(0)
    t = np.where(tot > 0, counts.argmax(0), -1)
    return tot, t


@pytest.mark.parametrize("n", [1, 2, 3, 6, 21])
def test_nsew_all_horizontal_start_is_north_above_south_below(n):
    # the all-horizontal start: every face in the upper half of the diamond is
    # covered by a north domino, every face in the lower half by a south one
    counts = O.domino_nsew(O.aztec(n), n % 2)
    inside = _aztec_faces(n).astype(bool)
    tot, t = _nsew_types(counts)
    assert np.array_equal(tot, inside.astype(np.uint32))
    ys = np.arange(2 * n)[:, None] * np.ones((1, 2 * n), dtype=int)
    assert np.all(t[inside & (ys >= n)] == 0)
    assert np.all(t[inside & (ys < n)] == 1)
    assert counts[2].sum() == 0 and counts[3].sum() == 0


def _rot180(st):
    # face (x, y) -> (2n-1-x, 2n-1-y); primal edges map Hz(x,y) -> Hz(W-2-x, H-1-y),
    # Vt(x,y) -> Vt(W-1-x, H-2-y)
    out = np.zeros_like(st)
    _, H, W = st.shape
    out[0, :, : W - 1] = st[0, ::-1, : W - 1][:, ::-1]
    out[1, : H - 1, :] = st[1, : H - 1, ::-1][::-1, :]
    return out


def _transpose(st):
    # reflection in the diagonal x <-> y: Hz(x,y) <-> Vt(y,x)
    return np.ascontiguousarray(np.stack([st[1].T, st[0].T]))


@pytest.mark.parametrize("n", [1, 2, 5, 12, 30])
def test_nsew_one_type_per_face_and_symmetries(n):
    inside = _aztec_faces(n).astype(bool)
    for seed in range(3):
        st = O.aztec_shuffle(n, seed, stream=1)
        counts = O.domino_nsew(st, n % 2)
        tot, t = _nsew_types(counts)
        # every face of the diamond carries exactly one type, nothing outside
        assert np.array_equal(tot, inside.astype(np.uint32))
        # a half turn keeps colours and swaps north/south and east/west
        r = _rot180(st)
        assert O.domino_check(r, inside) == 0
        cr = O.domino_nsew(r, n % 2)
        assert np.array_equal(cr[[1, 0, 3, 2]], counts[:, ::-1, ::-1])
        # the diagonal reflection maps north -> east, south -> west and back
        tr = _transpose(st)
        assert O.domino_check(tr, inside) == 0
        ct = O.domino_nsew(tr, n % 2)
        assert np.array_equal(ct[[2, 3, 0, 1]], counts.transpose(0, 2, 1))


def test_nsew_frozen_corners_carry_the_four_types():
    # on exact samples of order 30 the four corners of the diamond are frozen:
    # north brickwork at the top, south at the bottom, west on the left,
    # east on the right
    n = 30
    for seed in range(4):
        _, t = _nsew_types(O.domino_nsew(O.aztec_shuffle(n, seed, stream=2), n % 2))
        assert np.all(t[2 * n - 3:, n - 1:n + 1] == 0)       # top: faces (n-1..n, 2n-3..2n-1)
        assert np.all(t[:3, n - 1:n + 1] == 1)               # bottom
        assert np.all(t[n - 1:n + 1, 2 * n - 3:] == 2)       # right: east
        assert np.all(t[n - 1:n + 1, :3] == 3)               # left: west
