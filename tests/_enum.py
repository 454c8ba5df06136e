"""Brute-force helpers over the oracle: enumerate all states reachable by
single-site moves and build exact per-pass transition matrices.

Used only by the CPU tests that pin the oracle.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np

import oracle as O


def single_flips(lattice, st):
    """All states one elementary move away (every class, every rotatable site)."""
    out = []
    for p in range(O.PASSES[lattice]):
        codes = O.site_states(lattice, st, p)
        ys, xs = np.nonzero(codes)
        base = (codes == 2).astype(np.uint8)   # keep every site as it is ...
        for y, x in zip(ys, xs):
            dec = base.copy()
            dec[y, x] ^= 1                      # ... except this one
            nxt = st.copy()
            O.apply_pass(lattice, nxt, p, dec)
            out.append(nxt)
    return out


def enumerate_states(lattice, st0, limit=200000):
    """Breadth-first closure of st0 under elementary moves (Thurston)."""
    seen = {st0.tobytes(): 0}
    states = [st0.copy()]
    i = 0
    while i < len(states):
        for nxt in single_flips(lattice, states[i]):
            key = nxt.tobytes()
            if key not in seen:
                seen[key] = len(states)
                states.append(nxt)
                if len(states) > limit:
                    raise RuntimeError("state space too large")
        i += 1
    return states, seen


def pass_matrix(lattice, states, index, p, prob_up):
    """Exact transition matrix of one heat-bath pass over class p.

    prob_up(st, y, x) -> probability that a rotatable site goes UP.  Each
    rotatable class site decides independently (the cluster move of Sec. 1.1.3).
    """
    n = len(states)
    P = np.zeros((n, n), dtype=np.float64)
    for a, st in enumerate(states):
        codes = O.site_states(lattice, st, p)
        ys, xs = np.nonzero(codes)
        probs = [prob_up(st, y, x) for y, x in zip(ys, xs)]
        for choice in itertools.product((0, 1), repeat=len(ys)):
            pr = 1.0
            dec = np.zeros(codes.shape, dtype=np.uint8)
            for (y, x), c, q in zip(zip(ys, xs), choice, probs):
                dec[y, x] = c
                pr *= q if c else (1.0 - q)
            nxt = st.copy()
            O.apply_pass(lattice, nxt, p, dec)
            P[a, index[nxt.tobytes()]] += pr
    return P


def thresh_prob(t):
    """P(u < t) for u uniform on 32 bits."""
    return float(Fraction(int(t), 1 << 32))
