"""The allocation-free height entry point, tl_read_height_noalloc.

Some callers cannot allocate device memory at the moment they want the
height function: code running under a device-memory budget that forbids new
allocations, or a tight loop that must not pay the device-wide
synchronisation that cudaMalloc / cudaFree can cause.  tl_read_height_noalloc
serves them: it writes the same heights as tl_read_height into a device
buffer the caller already owns, and keeps its per-row scratch in one static
device array instead of memory it allocates.

Here it is called through the C-ABI, twice in a row and again after more
sweeps, and its output must equal tl_read_height's exactly (heights are
integers).  This file is collected last on purpose.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_07250_gb300 as T
    return T


def _chains(T, ctx):
    yield "aztec", T.Chain(ctx, T.Domain.aztec(150), seed=5, th=T.thresholds(scalar=1 << 31))
    ta, _ = T.lozenge_thresholds(0.9995)
    yield "hexagon", T.Chain(ctx, T.Domain.hexagon(60, 80, 70), seed=6, th=T.thresholds(scalar=ta))
    t16 = T.sixv_thresholds([1, 1, 1, 1, math.sqrt(2), math.sqrt(2)])
    yield "dwbc", T.Chain(ctx, T.Domain.dwbc(200), seed=7, th=T.thresholds(table16=t16))


def test_noalloc_height_matches_read_height(T):
    import torch
    ctx = T.Context(0)
    stream = torch.cuda.Stream()
    for name, ch in _chains(T, ctx):
        shape = ch.domain.height_shape
        ref = torch.empty(shape, dtype=torch.int32, device="cuda")
        got = torch.empty(shape, dtype=torch.int32, device="cuda")
        seen = []
        for rnd in range(2):
            ch.run(40, stream=stream)
            ch.read_height(ref, stream=stream)
            for call in range(2):            # two calls in a row share the static scratch
                got.fill_(-7)
                ch.read_height_noalloc(got, stream=stream)
                stream.synchronize()
                assert torch.equal(got, ref), "%s: round %d call %d differs" % (name, rnd, call)
            seen.append(got.cpu().numpy().copy())
        # the two rounds were at different states, so the scratch really was rewritten
        assert not np.array_equal(seen[0], seen[1]), name


def test_noalloc_height_rejects_host_buffers(T):
    ctx = T.Context(0)
    ch = T.Chain(ctx, T.Domain.aztec(20), seed=1, th=T.thresholds(scalar=1 << 31))
    host = np.zeros(ch.domain.height_shape, dtype=np.int32)
    with pytest.raises(T.TilingError) as e:
        ch.read_height_noalloc(host)
    assert e.value.code == T.TL_EINVAL


def test_noalloc_height_allocates_nothing(T):
    # after the first call, repeated calls leave the device's free memory
    # exactly where it was: nothing is allocated, not even lazily
    import torch
    ctx = T.Context(0)
    ch = T.Chain(ctx, T.Domain.aztec(300), seed=3, th=T.thresholds(scalar=1 << 31))
    ch.run(20)
    out = torch.empty(ch.domain.height_shape, dtype=torch.int32, device="cuda")
    ch.read_height_noalloc(out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        ch.read_height_noalloc(out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_height_rejects_too_many_segments(T):
    # a 6 x 65534 rectangle with a 2 x 4 notch cut from the middle of its top
    # edge: 65535 vertex rows, four of them split in two by the notch, so
    # 65539 height segments -- more than the static scratch holds
    ctx = T.Context(0)
    steps = ([0] * 6 + [1] * 65534 + [2] * 2 + [3] * 4 + [2] * 2 + [1] * 4 + [2] * 2 + [3] * 65534)
    dom = T.Domain.from_boundary(T.DOMINO, steps)
    ch = T.Chain(ctx, dom, seed=1, th=T.thresholds(scalar=1 << 31))
    import torch
    out = torch.empty(dom.height_shape, dtype=torch.int32, device="cuda")
    with pytest.raises(T.TilingError) as e:
        ch.read_height_noalloc(out)
    assert e.value.code == T.TL_EINVAL
    # the allocating call still serves it
    ref = ch.read_height()
    assert ref.shape == dom.height_shape
