"""The oracle reproduces its stored golden rollout (written by tests/golden/make_golden.py).

A regression fixture of the oracle: any change to the oracle's arithmetic that moves these
numbers must be justified by the passage or reading it implements."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_cube_floor_rollout_matches_golden():
    stored = np.loadtxt(os.path.join(HERE, "golden", "cube_floor_rollout.txt"))
    rows = make_golden.cube_floor_rollout()
    assert stored.shape == rows.shape
    assert np.allclose(rows, stored, rtol=1e-12, atol=1e-15)
