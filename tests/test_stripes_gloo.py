"""One chain split across ranks by rows (gloo on CPU): the partition, the
halo-exchange schedule and the row exchange of `stripes.py`.

Each rank advances only the rows it holds (its stripe and `halo` rows each
side), with the oracle's per-site draws keyed by absolute coordinates and
sweep, and exchanges boundary rows every `halo` passes.  Gathered, the owned
rows must equal the single-process oracle chain exactly, for any number of
ranks and any halo: which rows are sent, when, and that the random numbers do
not depend on the rank count.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SEED, STREAM, T_HALF = 5, 3, 1 << 31


def _pass_rows(O, st, sweep, slot, rows):
    """One heat-bath pass of colour `slot` (fixed order) on the sites of rows
    [a, b) only; every other site keeps its orientation."""
    _, H, W = st.shape
    a, b = rows
    Rp = ((W + 1) // 2 + 127) // 128 * 128
    states = O.site_states(O.DOMINO, st, slot)
    dec = (states == 2).astype(np.uint8)            # outside [a, b): keep
    ys, xs = np.nonzero(states)
    for y, x in zip(ys, xs):
        if a <= y < b:
            u = O.site_u(SEED, STREAM, sweep, slot, int(y) * Rp + (int(x) >> 1))
            dec[y, x] = 1 if u < T_HALF else 0
    O.apply_pass(O.DOMINO, st, slot, dec)


def _worker(rank, world, port, n, k, halo, out_dir):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_1804_07250_gb300 import stripes as S

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = O.aztec_shuffle(n, 1, stream=0)     # a disordered start: flips everywhere
        H = st.shape[1]
        bounds = S.partition(H, world, halo)
        rows = S.local_rows(bounds, rank, halo, H)
        state = torch.from_numpy(st)
        done = 0
        for hc in S.cycles(2 * k, halo):
            for _ in range(hc):
                sweep, slot = divmod(done, 2)
                arr = state.numpy()
                _pass_rows(O, arr, sweep, slot, rows)
                done += 1
            if done < 2 * k:
                S.exchange(state, bounds, rank, halo, dist)
        lo, hi = bounds[rank]
        np.save(os.path.join(out_dir, "r%d.npy" % rank), state.numpy()[:, lo:min(hi, H), :])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,halo", [(2, 4), (3, 2), (2, 6)])
def test_stripes_reproduce_the_single_chain(tmp_path, world, halo):
    import torch.multiprocessing as mp

    import oracle as O
    from paper_1804_07250_gb300 import stripes as S

    n, k = 12, 150
    mp.start_processes(_worker, args=(world, _free_port(), n, k, halo, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    parts = [np.load(tmp_path / ("r%d.npy" % r)) for r in range(world)]
    got = np.concatenate(parts, axis=1)
    want = O.aztec_shuffle(n, 1, stream=0)
    O.sweeps(O.DOMINO, want, seed=SEED, stream=STREAM, k=k, t_scalar=T_HALF)
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    # the bookkeeping itself
    b = S.partition(want.shape[1], world, halo)
    assert b[0][0] == 0 and b[-1][1] >= want.shape[1] and all(lo % 2 == 0 and hi - lo >= halo for lo, hi in b)
    assert sum(S.cycles(2 * k, halo)) == 2 * k


def test_partition_edges():
    from paper_1804_07250_gb300 import stripes as S
    assert S.partition(4097, 1, 8) == [(0, 4098)]
    b = S.partition(4097, 152, 8)
    assert len(b) == 152 and b[-1][1] == 4098 and min(hi - lo for lo, hi in b) >= 8
    with pytest.raises(ValueError):
        S.partition(20, 4, 8)
    assert S.local_rows(b, 0, 8, 4097)[0] == 0 and S.local_rows(b, 151, 8, 4097)[1] == 4097
    assert S.cycles(10, 4) == [4, 4, 2]
