"""The oracle reproduces its recorded regression results (tests/golden)."""
import os

import numpy as np

from tests.golden.make_golden import disc2d_history

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_disc2d_regression(oracle_lib):
    rows, l1, a = disc2d_history()
    ref = np.loadtxt(os.path.join(HERE, "disc2d_oracle.txt"))
    got = np.array(rows, float)
    assert np.allclose(got[:, :5], ref[:, :5], rtol=1e-12, atol=1e-15)
    assert np.array_equal(got[:, 5:], ref[:, 5:])
    a_ref = np.loadtxt(os.path.join(HERE, "disc2d_oracle_alpha20.txt"))
    assert np.abs(a - a_ref).max() < 1e-13
    with open(os.path.join(HERE, "disc2d_oracle.txt")) as f:
        l1_ref = float([ln for ln in f if ln.startswith("# L1")][0].split(":")[1])
    assert abs(l1 - l1_ref) <= 1e-12 * l1_ref
