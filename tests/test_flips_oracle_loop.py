"""The pass-by-pass oracle loop that counts rotations for the flip-counter
GPU test reproduces the oracle's own sweeps (no GPU)."""
import numpy as np

import oracle as O
from tests.test_gpu_flips import _oracle_flips_from


def test_oracle_pass_loop_is_the_oracle_chain():
    # the test's pass-by-pass loop reproduces the oracle's own sweeps
    st = O.aztec(10)
    a = st.copy()
    _oracle_flips_from(O.DOMINO, a, seed=5, stream=1, sweep0=0, k=6, t=1 << 31)
    b = st.copy()
    O.sweeps(O.DOMINO, b, seed=5, stream=1, k=6, t_scalar=1 << 31)
    assert np.array_equal(a, b)
