"""Failure path of the bounded device waits, without a GPU fault.

The resident kernels wait for their neighbours' boundary rows and the
batched kernel for each tile's bulk copy; every such wait is bounded and,
when it gives up, raises a status word, stops the kernel and surfaces as
TL_ETIMEOUT.  Here the status word is raised by the host (the library's test
hook) so that the next launch stops at its first wait point exactly as if a
wait had run out: the error must be reported, promptly, and the chain or
batch must be usable again, bit-exact against the oracle, after it is reset
or rewritten.  Nothing here faults, traps or hangs the GPU: every wait
returns.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle as O
from tests.test_gpu_batch import _make, _oracle, _specs

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


@pytest.mark.parametrize("kernel,scalar", [(3, T_HALF), (2, T_HALF), (2, 0x6A09E667)])
def test_resident_wait_gives_up_and_chain_recovers(T, ctx, kernel, scalar):
    n = 150
    dom = T.Domain.aztec(n)
    ch = T.Chain(ctx, dom, seed=9, stream_id=1, th=T.thresholds(scalar=scalar))
    ch.set_plan(kernel)
    assert ch.plan()["kernel"] == kernel
    ch.run(20)
    ch.sync()
    # raised status: the launch stops at its first boundary exchange
    ch.debug_raise_status()
    t0 = time.perf_counter()
    ch.run(200)
    with pytest.raises(T.TilingError) as e:
        ch.sync()
    assert e.value.code == T.TL_ETIMEOUT
    assert time.perf_counter() - t0 < 1.0        # no wait ran to its 2 s limit
    ch.sync()                                    # the word was cleared with the report
    # recovery 1: reset to the start, then bit-exact against the oracle
    ch.reset()
    ring = ch.run_hashed(60)
    st = O.aztec(n)
    want = O.sweeps(O.DOMINO, st, seed=9, stream=1, k=60, t_scalar=scalar, want_hashes=True)
    assert np.array_equal(ring, want)
    assert np.array_equal(ch.read_state(), st)
    # recovery 2: fail again, then rewrite the state at a chosen sweep index
    ch.debug_raise_status()
    ch.run(100)
    with pytest.raises(T.TilingError) as e:
        ch.sync()
    assert e.value.code == T.TL_ETIMEOUT
    ch.seek(60)
    ch.write_state(st)
    ch.run(40)
    ch.sync()
    O.sweeps(O.DOMINO, st, seed=9, stream=1, sweep0=60, k=40, t_scalar=scalar)
    assert np.array_equal(ch.read_state(), st)


def test_per_pass_kernel_has_no_waits(T, ctx):
    ch = T.Chain(ctx, T.Domain.aztec(20), seed=1, th=T.thresholds(scalar=T_HALF))
    ch.set_plan(1)
    with pytest.raises(T.TilingError) as e:
        ch.debug_raise_status()
    assert e.value.code == T.TL_EUNSUPPORTED


def test_batch_wait_gives_up_and_batch_recovers(T, ctx):
    import torch
    specs = _specs()
    chains = [_make(T, ctx, sp, 500 + i) for i, sp in enumerate(specs)]
    b = T.Batch(ctx, chains)
    stream = torch.cuda.Stream()
    b.run(8, stream=stream)
    stream.synchronize()
    b.hashes()
    b.debug_raise_status()
    t0 = time.perf_counter()
    b.run(16, stream=stream)
    stream.synchronize()
    with pytest.raises(T.TilingError) as e:
        b.hashes()
    assert e.value.code == T.TL_ETIMEOUT
    assert time.perf_counter() - t0 < 1.0
    # the chains are undefined now: take them out, reset them, batch them again
    for ch in list(chains):
        b.remove(ch)
        ch.reset()
    b2 = T.Batch(ctx, chains)
    b2.run(24, stream=stream)
    stream.synchronize()
    hb = b2.hashes()
    for i, (sp, ch) in enumerate(zip(specs, chains)):
        st = _oracle(sp, 500 + i, 24)
        assert int(hb[i]) == O.state_hash(st), "chain %d" % i
        assert np.array_equal(ch.read_state(), st), "chain %d" % i
