"""The oracle against its stored output for the 1S0 Yamaguchi workload
(tests/golden/yamaguchi_1s0_nwp32.txt, written by tests/golden/make_golden.py
from the oracle): a regression pin that catches any change to the oracle's
arithmetic on this case."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_yamaguchi():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    e, delta, sigma = make_golden.yamaguchi()
    ref = np.loadtxt(os.path.join(HERE, "golden", "yamaguchi_1s0_nwp32.txt"))
    assert ref.shape == (64, 3)
    assert np.array_equal(ref[:, 0], e)
    assert np.max(np.abs(delta - ref[:, 1])) <= 1e-9          # degrees
    assert np.max(np.abs(sigma - ref[:, 2]) / ref[:, 2]) <= 1e-11
