"""Stored oracle values (tests/golden/, written by tests/golden/make_golden.py
from the oracle alone): the oracle must keep reproducing them, and the values of
the steady zonal flow must match the flow's closed form."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2605_01313_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402


def load(name):
    rows = np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)
    idx = rows[:, 0].astype(np.int64)
    lon, colat = rows[:, 1], rows[:, 2]
    vals = rows[:, 3::2] + 1j * rows[:, 4::2]          # (P, F)
    return idx, lon, colat, vals.T


@pytest.mark.parametrize("name", sorted(make_golden.FIXTURES))
def test_oracle_reproduces_stored_values(name):
    idx, lon, colat, stored = load(name)
    c, lon_now, colat_now, idx_now = make_golden.FIXTURES[name][0]()
    # the seeded inputs are unchanged ...
    assert np.array_equal(idx, idx_now)
    assert np.array_equal(lon, lon_now) and np.array_equal(colat, colat_now)
    # ... and the oracle's arithmetic too (libm may differ in the last unit
    # across machines: 1e-14 of the largest value)
    v = oracle.evaluate(c, lon, colat).reshape(stored.shape)
    assert np.max(np.abs(v - stored)) <= 1e-14 * np.max(np.abs(stored))


def test_stored_zonal_flow_matches_closed_form():
    """The stored (h, u, v) of the tilted steady zonal flow against its pointwise
    formulas (Sec. 6), anywhere on the doubled torus (the wind components change
    sign through the pole, which the formulas carry by themselves)."""
    _, lon, colat, stored = load("tc2_oracle_values.txt")
    exact = np.stack(synth.zonal_flow_values(lon, colat, math.pi / 2 - 0.05))
    for f in range(3):
        scale = np.max(np.abs(exact[f]))
        assert np.max(np.abs(stored[f].real - exact[f])) <= 1e-13 * scale
        assert np.max(np.abs(stored[f].imag)) <= 1e-13 * scale
