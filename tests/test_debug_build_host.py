"""The bounds-checked build compiles and loads on the host (no GPU call).

`_build.py --debug` builds libtiling_debug.so with -DTL_DEBUG; the binding
loads it when TL_DEBUG=1.  Its tl_debug_build answers 1 (the normal build's
answers 0), and it exports every symbol the header declares.  The checks
themselves run on the GPU (tests/test_gpu_debug_build.py).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_compiles_and_loads():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    subprocess.run([sys.executable, os.path.join(ROOT, "paper_1804_07250_gb300", "_build.py"), "--debug"],
                   cwd=ROOT, check=True, timeout=900, capture_output=True)
    code = (
        "import paper_1804_07250_gb300 as T\n"
        "assert T.LIB_PATH.endswith('libtiling_debug.so'), T.LIB_PATH\n"
        "assert T.debug_build()\n"
        "assert all(hasattr(T.lib(), n) for n in T.EXPORTED)\n"
    )
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, env={**os.environ, "TL_DEBUG": "1"}, check=True,
                   timeout=300)


def test_normal_build_answers_zero():
    import paper_1804_07250_gb300 as T
    if T.DEBUG_BUILD:
        pytest.skip("running under the checked build")
    assert not T.debug_build()
