"""The bounds-checked build (libtiling_debug.so, -DTL_DEBUG).

Its index checks record a failure in a device word and skip the access
instead of faulting.  Here the checked library is built, its self-test must
report exactly the one out-of-range check it makes, and a selection of the
parity tests (every kernel: register and shared-memory resident, per-pass,
batched, shuffling, heights, regions and random order) runs against it in a
child process: bit-exact against the oracle as in the normal build, with no
failed check after any test (the autouse fixture in conftest.py).
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    "tests/test_gpu_regdom.py::test_aztec_halos",
    "tests/test_gpu_regdom.py::test_regions",
    "tests/test_gpu_regdom.py::test_random_pass_order",
    "tests/test_gpu_regdom.py::test_density_and_nsew",
    "tests/test_gpu_parity.py::test_resident_kernel_halos",
    "tests/test_gpu_parity.py::test_resident_threshold_kinds",
    "tests/test_gpu_parity.py::test_global_per_pass_kernel",
    "tests/test_gpu_parity.py::test_height_matches_oracle",
    "tests/test_gpu_parity.py::test_density_matches_oracle",
    "tests/test_gpu_batch.py::test_batch_matches_alone_and_oracle",
    "tests/test_gpu_shuffle_arctic.py::test_shuffle_matches_oracle",
    "tests/test_gpu_regions_cftp.py::test_random_order_parity",
]


@pytest.fixture(scope="module")
def debug_env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if os.environ.get("TL_DEBUG") == "1":
        pytest.skip("already running under the checked build")
    sys.path.insert(0, ROOT)
    from paper_1804_07250_gb300 import _build
    _build.build(debug=True)
    return {**os.environ, "TL_DEBUG": "1"}


def test_selftest_reports_one_failure(debug_env):
    code = (
        "import paper_1804_07250_gb300 as T\n"
        "assert T.debug_build()\n"
        "T.debug_checks(clear=True)\n"
        "T.debug_selftest()\n"
        "r = T.debug_checks(clear=True)\n"
        "assert r == {'failures': 1, 'id': 999, 'index': 5, 'bound': 3}, r\n"
        "assert T.debug_checks()['failures'] == 0\n"
    )
    subprocess.run([sys.executable, "-c", code], env=debug_env, cwd=ROOT, check=True, timeout=300)


def test_parity_selection_runs_clean(debug_env):
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *SELECTION], env=debug_env, cwd=ROOT, capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]


def test_normal_build_has_no_checks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if os.environ.get("TL_DEBUG") == "1":
        pytest.skip("running under the checked build")
    import paper_1804_07250_gb300 as T
    assert not T.debug_build()
    with pytest.raises(T.TilingError) as e:
        T.debug_checks()
    assert e.value.code == T.TL_EUNSUPPORTED
