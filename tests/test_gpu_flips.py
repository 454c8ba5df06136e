"""Accepted-flip counters: the number of site rotations a chain performed
must equal the count the oracle's own pass-by-pass run gives (a site counts
when a pass leaves it in the other orientation), on every single-chain
kernel."""
from __future__ import annotations

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


@pytest.mark.parametrize("kind,kernel,t", [("aztec", 3, 1 << 31), ("aztec", 2, 1 << 31), ("aztec", 1, 1 << 31),
                                           ("aztec", 2, 0x6A09E667), ("aztec", 1, 0x6A09E667),
                                           ("hex", 2, 0x7FF80000), ("hex", 1, 0x7FF80000)])
def test_flip_counter_matches_oracle(T, kind, kernel, t):
    ctx = T.Context(0)
    if kind == "aztec":
        dom, st, lat = T.Domain.aztec(24), O.aztec(24), O.DOMINO
    else:
        dom, st, lat = T.Domain.hexagon(12, 10, 14), O.hexagon(12, 10, 14), O.LOZENGE
    ch = T.Chain(ctx, dom, seed=31, stream_id=2, th=T.thresholds(scalar=t))
    ch.set_plan(kernel)
    ch.run(3)                      # not counted
    ch.count_flips(True)
    ch.run(10)
    ch.run(17)
    got = ch.flips
    # the oracle from the same start: 3 uncounted sweeps, then 27 counted
    O.sweeps(lat, st, seed=31, stream=2, k=3, t_scalar=t)
    ref = st.copy()
    want = _oracle_flips_from(lat, ref, seed=31, stream=2, sweep0=3, k=27, t=t)
    assert got == want
    assert np.array_equal(ch.read_state(), ref)
    ch.count_flips(False)
    ch.run(5)
    assert ch.flips == want          # stopped, not reset


def _oracle_flips_from(lat, st, *, seed, stream, sweep0, k, t):
    _, H, W = st.shape
    npar = 3 if lat == O.LOZENGE else 2
    Rp = ((W + npar - 1) // npar + 127) // 128 * 128
    flips = 0
    for sweep in range(sweep0, sweep0 + k):
        for p in range(O.PASSES[lat]):
            states = O.site_states(lat, st, p)
            dec = np.zeros_like(states)
            ys, xs = np.nonzero(states)
            for y, x in zip(ys, xs):
                u = O.site_u(seed, stream, sweep, p, int(y) * Rp + int(x) // npar)
                dec[y, x] = 1 if u < t else 0
                flips += int((states[y, x] == 2) != bool(dec[y, x]))
            O.apply_pass(lat, st, p, dec)
    return flips
