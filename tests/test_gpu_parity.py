"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

The chain is a deterministic function of (domain, start, thresholds, seed,
stream, sweep index), so the packed GPU state must equal the oracle's state
bit for bit after every sweep.  Sizes span several 128-site groups with a
ragged tail, the smallest domains, extreme thresholds, and the full benchmark
sizes (sampled: the first sweeps in full, then invariants).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SQ2 = [1, 1, 1, 1, math.sqrt(2), math.sqrt(2)]


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


def _domain(T, kind, args):
    return {"aztec": T.Domain.aztec, "rect": T.Domain.rect, "hex": T.Domain.hexagon,
            "dwbc": T.Domain.dwbc}[kind](*args)


def _oracle_state(kind, args):
    return {"aztec": O.aztec, "rect": O.rect, "hex": O.hexagon, "dwbc": O.dwbc}[kind](*args)


def _lat(kind):
    return {"aztec": O.DOMINO, "rect": O.DOMINO, "hex": O.LOZENGE, "dwbc": O.SIXV}[kind]


def _run_pair(T, ctx, kind, args, *, seed, stream=0, k, kernel=0, spl=0, halo=0, threads=0,
              npre=0, scalar=None, site=None, w6=None, hashed=True):
    dom = _domain(T, kind, args)
    lat = _lat(kind)
    if lat == O.SIXV:
        t16 = O.sixv_thresholds(w6)
        th = T.thresholds(table16=t16)
        okw = dict(t16=t16)
    elif site is not None:
        th = T.thresholds(site=site)
        okw = dict(t_site=site)
    else:
        th = T.thresholds(scalar=scalar)
        okw = dict(t_scalar=scalar)
    ch = T.Chain(ctx, dom, seed=seed, stream_id=stream, th=th)
    if kernel or spl or halo or threads or npre:
        ch.set_plan(kernel, spl, halo, threads, npre)
    st = _oracle_state(kind, args)
    if hashed:
        ring = ch.run_hashed(k)
        ohash = O.sweeps(lat, st, seed=seed, stream=stream, k=k, want_hashes=True, **okw)
        bad = np.nonzero(ring != ohash)[0]
        assert bad.size == 0, "first mismatch at sweep %d" % bad[0]
    else:
        ch.run(k)
        O.sweeps(lat, st, seed=seed, stream=stream, k=k, **okw)
    ch.sync()
    got = ch.read_state()
    assert np.array_equal(got, st)
    assert ch.state_hash() == O.state_hash(st)
    assert ch.sweep == k
    return ch, st


# ---------------------------------------------------------------------------
# Bit-exact trajectories
# ---------------------------------------------------------------------------
def test_aztec32_uniform_every_sweep_full_length(T, ctx):
    # Aztec diamond n = 32, seed 1, t = 2^31, 10^4 sweeps, hash after every sweep
    _run_pair(T, ctx, "aztec", (32,), seed=1, k=10_000, scalar=1 << 31)


@pytest.mark.parametrize("kind,args", [
    ("aztec", (1,)), ("aztec", (2,)), ("aztec", (63,)), ("aztec", (64,)), ("aztec", (129,)),
    ("rect", (2, 2)), ("rect", (300, 7)), ("rect", (255, 8)), ("rect", (7, 40)),
])
def test_domino_uniform_sizes(T, ctx, kind, args):
    _run_pair(T, ctx, kind, args, seed=12345, stream=3, k=60, scalar=1 << 31)


@pytest.mark.parametrize("t", [0, 1, (1 << 31) - 1, (1 << 31) + 1, 0xC0000000, 0xFFFFFFFF, 123456789])
def test_domino_scalar_thresholds(T, ctx, t):
    _run_pair(T, ctx, "aztec", (40,), seed=99, k=30, scalar=t)


@pytest.mark.parametrize("n", [5, 37, 100])
def test_domino_edge_weights(T, ctx, n):
    rng = np.random.default_rng(n)
    W = 2 * n + 1
    w = np.exp(0.5 * rng.standard_normal((2, W, W)))
    t = O.domino_thresholds(w)
    _run_pair(T, ctx, "aztec", (n,), seed=3, stream=n, k=40, site=t)


@pytest.mark.parametrize("abc", [(1, 1, 1), (2, 3, 4), (20, 9, 33), (150, 200, 130)])
def test_lozenge_q(T, ctx, abc):
    ta, _ = O.lozenge_thresholds(0.9995)
    _run_pair(T, ctx, "hex", abc, seed=11, k=40, scalar=ta)


def test_lozenge_site_thresholds(T, ctx):
    a, b, c = 30, 41, 25
    rng = np.random.default_rng(7)
    st = O.hexagon(a, b, c)
    t = rng.integers(0, 1 << 32, size=st.shape[1:], dtype=np.uint64).astype(np.uint32)
    _run_pair(T, ctx, "hex", (a, b, c), seed=5, k=40, site=t)


@pytest.mark.parametrize("N", [2, 3, 4, 11, 260, 301])
def test_sixv_dwbc_sqrt2(T, ctx, N):
    _run_pair(T, ctx, "dwbc", (N,), seed=11, k=50, w6=SQ2)


@pytest.mark.parametrize("w6", [[1] * 6, [1, 1, 1, 1, math.sqrt(8), math.sqrt(8)],
                                [0.7, 1.3, 0.4, 1.9, 1.1, 0.6]])
def test_sixv_weights(T, ctx, w6):
    _run_pair(T, ctx, "dwbc", (130,), seed=2, stream=9, k=40, w6=w6)


# ---------------------------------------------------------------------------
# Both kernel families, several halo depths and launch splits
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,args", [("aztec", (70,)), ("hex", (40, 50, 45)), ("dwbc", (120,))])
def test_global_per_pass_kernel(T, ctx, kind, args):
    kw = dict(w6=SQ2) if kind == "dwbc" else dict(scalar=(1 << 31) if kind == "aztec" else 0x7FF80000)
    _run_pair(T, ctx, kind, args, seed=17, k=30, kernel=1, **kw)


@pytest.mark.parametrize("halo", [1, 2, 3, 5, 8, 13])
@pytest.mark.parametrize("kind,args", [("aztec", (90,)), ("hex", (60, 70, 50)), ("dwbc", (150,))])
def test_resident_kernel_halos(T, ctx, kind, args, halo):
    kw = dict(w6=SQ2) if kind == "dwbc" else dict(scalar=(1 << 31) if kind == "aztec" else 0x7FF80000)
    _run_pair(T, ctx, kind, args, seed=23, k=25, kernel=2, halo=halo, **kw)


@pytest.mark.parametrize("threads", [512, 1024])
@pytest.mark.parametrize("npre", [1, 2, 4, 8])
@pytest.mark.parametrize("kind,args", [("aztec", (90,)), ("hex", (60, 70, 50)), ("dwbc", (150,))])
def test_resident_kernel_threads_npre(T, ctx, kind, args, threads, npre):
    kw = dict(w6=SQ2) if kind == "dwbc" else dict(scalar=(1 << 31) if kind == "aztec" else 0x7FF80000)
    _run_pair(T, ctx, kind, args, seed=29, k=20, kernel=2, threads=threads, npre=npre, **kw)


@pytest.mark.parametrize("npre", [1, 8, 16])
@pytest.mark.parametrize("case", ["aztec_t", "aztec_site", "hex", "hex_site", "dwbc", "dwbc_w", "dwbc_flat"])
def test_resident_threshold_kinds(T, ctx, case, npre):
    # every threshold form through the resident kernel: scalar and per-site
    # (random 32-bit values), and six-vertex tables in count form (c = sqrt 2,
    # all weights equal) and general form (random weights)
    rng = np.random.default_rng([41, npre])
    if case.startswith("aztec"):
        kind, args = "aztec", (110,)
    elif case.startswith("hex"):
        kind, args = "hex", (70, 55, 64)
    else:
        kind, args = "dwbc", (170,)
    if case.endswith("_site"):
        shape = _oracle_state(kind, args).shape[1:]
        kw = dict(site=rng.integers(0, 1 << 32, size=shape, dtype=np.uint64).astype(np.uint32))
    elif kind == "dwbc":
        kw = dict(w6={"dwbc": SQ2, "dwbc_flat": [1.0] * 6,
                      "dwbc_w": list(np.exp(0.7 * rng.standard_normal(6)))}[case])
    else:
        kw = dict(scalar=0x7FF80000 if kind == "hex" else 0x9E3779B9)
    _run_pair(T, ctx, kind, args, seed=43, stream=5, k=24, kernel=2, npre=npre, **kw)


@pytest.mark.parametrize("spl", [1, 4, 7])
def test_resident_kernel_launch_splits(T, ctx, spl):
    _run_pair(T, ctx, "aztec", (128,), seed=31, k=30, kernel=2, spl=spl, scalar=1 << 31)


def test_resident_weighted(T, ctx):
    n = 150
    rng = np.random.default_rng(1)
    w = np.exp(0.5 * rng.standard_normal((2, 2 * n + 1, 2 * n + 1)))
    _run_pair(T, ctx, "aztec", (n,), seed=3, stream=77, k=30, kernel=2, site=O.domino_thresholds(w))


def test_resident_density_matches_global(T, ctx):
    dom = T.Domain.aztec(100)
    out = []
    for kernel in (1, 2):
        ch = T.Chain(ctx, dom, seed=12, th=T.thresholds(scalar=1 << 31))
        ch.set_plan(kernel)
        ch.density_begin(stride=7, burn_in=20)
        ch.run(33)
        ch.run(60)
        ch.sync()
        d, n = ch.read_density()
        out.append((d, n, ch.state_hash()))
    assert out[0][1] == out[1][1] == (93 - 20) // 7 + 1
    assert np.array_equal(out[0][0], out[1][0]) and out[0][2] == out[1][2]


def test_results_do_not_depend_on_how_sweeps_are_split(T, ctx):
    dom = T.Domain.aztec(50)
    a = T.Chain(ctx, dom, seed=8, th=T.thresholds(scalar=1 << 31))
    b = T.Chain(ctx, dom, seed=8, th=T.thresholds(scalar=1 << 31))
    a.run(100)
    for k in (1, 2, 3, 7, 87):
        b.run(k)
    assert a.state_hash() == b.state_hash()
    c = T.Chain(ctx, dom, seed=9, th=T.thresholds(scalar=1 << 31))
    c.run(100)
    assert c.state_hash() != a.state_hash()


# ---------------------------------------------------------------------------
# Full benchmark sizes on the default plan: every sweep of the first 1,000
# hashed and compared, then the whole state
# ---------------------------------------------------------------------------
def test_aztec2048_first_1000_sweeps(T, ctx):
    _run_pair(T, ctx, "aztec", (2048,), seed=7, k=1000, scalar=1 << 31, hashed=True)


def test_hexagon1024_first_1000_sweeps(T, ctx):
    ta, _ = O.lozenge_thresholds(0.9995)
    _run_pair(T, ctx, "hex", (1024, 1024, 1024), seed=11, k=1000, scalar=ta)


def test_dwbc2048_first_1000_sweeps(T, ctx):
    _run_pair(T, ctx, "dwbc", (2048,), seed=11, k=1000, w6=SQ2)


def test_long_run_crosses_launch_splits(T, ctx):
    # 2 x 10^5 sweeps on the default resident plan: one launch holds at most
    # 60,000 exchange cycles (16-bit cycle tags), so the run is split into
    # launches and tens of thousands of boundary exchanges take place; every
    # sweep's hash and the final state must equal the oracle's
    _run_pair(T, ctx, "aztec", (64,), seed=5, stream=2, k=200_000, kernel=2, scalar=1 << 31, hashed=True)


# ---------------------------------------------------------------------------
# Observables
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,args", [("aztec", (45,)), ("rect", (33, 20)), ("hex", (17, 23, 30)),
                                       ("dwbc", (70,))])
def test_height_matches_oracle(T, ctx, kind, args):
    lat = _lat(kind)
    kw = dict(w6=SQ2) if lat == O.SIXV else dict(scalar=1 << 31)
    ch, st = _run_pair(T, ctx, kind, args, seed=21, k=25, hashed=False, **kw)
    h = ch.read_height()
    ho, bad = O.height(lat, st)
    assert bad == 0
    assert np.array_equal(h, ho)


@pytest.mark.parametrize("n,kernel", [(20, 0), (21, 0), (64, 2), (45, 1)])
def test_density_matches_oracle(T, ctx, n, kernel):
    # edge densities and the per-face north/south/east/west densities equal
    # the oracle's counts divided by the number of samples
    dom = T.Domain.aztec(n)
    ch = T.Chain(ctx, dom, seed=4, th=T.thresholds(scalar=1 << 31))
    if kernel:
        ch.set_plan(kernel)
    ch.density_begin(stride=3, burn_in=10)
    ch.run(17)
    ch.run(40)
    dens, samples = ch.read_density()
    st = O.aztec(n)
    counts = np.zeros(st.shape, dtype=np.uint32)
    ncounts = np.zeros((4, 2 * n, 2 * n), dtype=np.uint32)
    nsamp = 0
    for s in range(57):
        O.sweeps(O.DOMINO, st, seed=4, sweep0=s, k=1, t_scalar=1 << 31)
        done = s + 1
        if done >= 10 and (done - 10) % 3 == 0:
            O.accumulate(st, counts)
            O.domino_nsew(st, n % 2, ncounts)
            nsamp += 1
    assert samples == nsamp
    assert np.array_equal(dens, counts / nsamp)
    nsew = ch.read_nsew()
    assert nsew.shape == ncounts.shape
    assert np.array_equal(np.rint(nsew * nsamp).astype(np.uint32), ncounts)
    np.testing.assert_allclose(nsew, ncounts / nsamp, rtol=0, atol=1e-15)
    # every domain face is covered by exactly one domino type per sample
    faces = nsew.sum(0)
    W = 2 * n
    for y in range(W):
        for x in range(W):
            inside = abs(x + 0.5 - n) + abs(y + 0.5 - n) <= n
            assert faces[y, x] == pytest.approx(1.0 if inside else 0.0, abs=1e-12)


def test_read_write_state_round_trip_and_validation(T, ctx):
    dom = T.Domain.hexagon(9, 8, 7)
    ch = T.Chain(ctx, dom, seed=1, th=T.thresholds(scalar=1 << 31))
    ch.run(30)
    s = ch.read_state()
    ch2 = T.Chain(ctx, dom, seed=1, th=T.thresholds(scalar=1 << 31), init=s)
    assert ch2.state_hash() == ch.state_hash()
    bad = s.copy()
    bad[0, 5, 5] ^= 1
    with pytest.raises(T.TilingError) as e:
        ch.write_state(bad)
    assert e.value.code == T.TL_EINVAL
    ch.write_state(O.hexagon(9, 8, 7))
    assert ch.state_hash() == O.state_hash(O.hexagon(9, 8, 7))


def test_device_buffers(T, ctx):
    import torch
    dom = T.Domain.aztec(30)
    ch = T.Chain(ctx, dom, seed=5, th=T.thresholds(scalar=1 << 31))
    stream = torch.cuda.Stream()
    ch.run(10, stream=stream)
    out = torch.zeros(dom.canon_shape, dtype=torch.uint8, device="cuda")
    ch.read_state(out, stream=stream)
    hbuf = torch.zeros(1, dtype=torch.int64, device="cuda")
    ch.state_hash(out=hbuf, stream=stream)
    stream.synchronize()
    st = O.aztec(30)
    O.sweeps(O.DOMINO, st, seed=5, k=10, t_scalar=1 << 31)
    assert np.array_equal(out.cpu().numpy(), st)
    assert int(hbuf.cpu().numpy().view(np.uint64)[0]) == O.state_hash(st)


@pytest.mark.parametrize("threads", [0, 512, 1024])
def test_resident_wide_domain_pass_capacity(T, ctx, threads):
    # a wide, short domain whose passes hold between 512 and 1024 groups per
    # CTA: more than the single-plane domino update takes, so the plan must
    # fall back to the general update with either thread count
    _run_pair(T, ctx, "rect", (8000, 30), seed=61, k=10, kernel=2, threads=threads, scalar=1 << 31)


@pytest.mark.parametrize("kind,args,kernel", [("aztec", (100,), 2), ("hex", (40, 50, 30), 2), ("hex", (40, 50, 30), 1),
                                               ("dwbc", (90,), 2)])
def test_density_counts_many_samples(T, ctx, kind, args, kernel):
    # one sample every sweep for 300 sweeps: the counters carry through nine
    # bit planes; counts must equal the oracle's exactly
    dom = _domain(T, kind, args)
    lat = _lat(kind)
    if lat == O.SIXV:
        t16 = O.sixv_thresholds(SQ2)
        th, okw = T.thresholds(table16=t16), dict(t16=t16)
    else:
        th, okw = T.thresholds(scalar=0x70000000), dict(t_scalar=0x70000000)
    ch = T.Chain(ctx, dom, seed=8, th=th)
    ch.set_plan(kernel)
    ch.density_begin(stride=1, burn_in=0)
    ch.run(300)
    dens, samples = ch.read_density()
    st = _oracle_state(kind, args)
    counts = np.zeros(st.shape, dtype=np.uint32)
    for s in range(300):
        O.sweeps(lat, st, seed=8, sweep0=s, k=1, **okw)
        O.accumulate(st, counts)
    assert samples == 300
    assert np.array_equal(np.rint(dens * 300).astype(np.uint32), counts)


def _reject(T, ch, bad):
    with pytest.raises(T.TilingError) as e:
        ch.write_state(bad)
    assert e.value.code == T.TL_EINVAL
    return str(e.value)


@pytest.mark.parametrize("where", ["host", "device"])
def test_write_state_rejects_every_kind(T, ctx, where):
    # the device validation rejects what the host validation of
    # tl_chain_create rejects, for every lattice and kind of failure, and
    # leaves the chain's state as it was
    import torch

    def put(a):
        return a if where == "host" else torch.from_numpy(a).cuda()

    cases = []
    st = O.aztec(12)
    b = st.copy(); b[0, 3, 7] = 2; cases.append(("aztec", (12,), st, b, "byte"))
    b = st.copy(); b[0, 12, 12] ^= 1; cases.append(("aztec", (12,), st, b, "face"))
    b = st.copy(); b[0, 5, st.shape[2] - 1] = 1; cases.append(("aztec", (12,), st, b, "edge outside"))
    hx = O.hexagon(6, 7, 5)
    b = hx.copy(); b[1, 4, 4] ^= 1; cases.append(("hexagon", (6, 7, 5), hx, b, "lozenge"))
    dw = O.dwbc(9)
    b = dw.copy(); b[0, 4, 4] ^= 1; cases.append(("dwbc", (9,), dw, b, "six-vertex"))
    b = dw.copy(); b[1, 0, 3] ^= 1; cases.append(("dwbc", (9,), dw, b, "six-vertex"))
    b = dw.copy(); b[0, 0, dw.shape[2] - 1] = 1; cases.append(("dwbc", (9,), dw, b, "six-vertex"))
    for kind, args, good, bad, word in cases:
        dom = getattr(T.Domain, kind)(*args)
        th = T.thresholds(table16=O.sixv_thresholds([1] * 6)) if kind == "dwbc" else T.thresholds(scalar=1 << 31)
        ch = T.Chain(ctx, dom, seed=2, th=th)
        ch.run(7)
        before = ch.state_hash()
        with pytest.raises(T.TilingError):
            T.Chain(ctx, dom, seed=2, th=th, init=bad)       # host validation
        msg = _reject(T, ch, put(bad))                       # device validation
        assert word in msg, (kind, msg)
        assert ch.state_hash() == before
        ch.write_state(put(good))
        assert ch.state_hash() == O.state_hash(good)
