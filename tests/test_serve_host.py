"""Host side of the serving loop: the synthetic request mix (Poisson
arrivals, a third of each domain kind, weights half uniform, sweeps
log-uniform) and the device footprint a job is admitted against.  Domains
are built on the host only; no GPU."""
import math

import numpy as np
import pytest

T = pytest.importorskip("paper_1804_07250_gb300")
serve = pytest.importorskip("paper_1804_07250_gb300.serve")


def test_request_mix_is_seeded_and_in_range():
    a = serve.make_requests(3000, 200.0, seed=5)
    b = serve.make_requests(3000, 200.0, seed=5)
    assert a == b
    assert serve.make_requests(50, 200.0, seed=6) != a[:50]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals: mean gap 1 / rate, coefficient of variation 1
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.06
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08
    kinds = [r.kind for r in a]
    for k in ("aztec", "hexagon", "dwbc"):
        assert abs(kinds.count(k) / len(a) - 1 / 3) < 0.04
    assert abs(sum(r.weights == "lognormal" for r in a) / len(a) - 0.5) < 0.04
    for r in a:
        if r.kind == "aztec":
            assert len(r.size) == 1 and 32 <= r.size[0] <= 2048
        elif r.kind == "hexagon":
            assert len(r.size) == 3 and all(16 <= s <= 512 for s in r.size)
        else:
            assert len(r.size) == 1 and 32 <= r.size[0] <= 1024
        assert 1000 <= r.sweeps <= 100_000
    # sweeps log-uniform: log10 spread evenly over [3, 5]
    lg = np.log10([r.sweeps for r in a])
    assert abs(lg.mean() - 4.0) < 0.05
    assert abs(np.mean(lg < 3.5) - 0.25) < 0.04


@pytest.mark.parametrize("dom", [lambda: T.Domain.aztec(100), lambda: T.Domain.hexagon(40, 50, 60),
                                 lambda: T.Domain.dwbc(90)])
def test_footprint_covers_the_buffers(dom):
    d = dom()
    info = d.info
    plain = serve.footprint(d, False)
    assert plain >= 3 * info.packed_bytes + info.canon_bytes + 4 * info.height_count
    if info.lattice != 2:
        # per-site weights add their threshold planes and the int32 staging
        assert serve.footprint(d, True) >= plain + 4 * info.site_box


def test_footprint_grows_with_the_domain():
    f = [serve.footprint(T.Domain.aztec(n), True) for n in (64, 128, 256, 512)]
    assert all(b > a for a, b in zip(f, f[1:]))
    # quadratic in the order: doubling n multiplies the bytes by about 4
    r = f[-1] / f[-2]
    assert 3.5 < r < 4.5
    assert math.isfinite(r)
