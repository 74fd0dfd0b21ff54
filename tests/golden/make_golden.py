"""Writes the stored expected values under tests/golden/ from the oracle alone.

The paper prints no value of Eq. 5.3 at given points that these fixtures could
hold, so each fixture is the FP64 oracle's own output on a seeded input from
paper_2605_01313_gb300.synth (input generation only), written once by this
script: tests/test_golden.py recomputes them and fails on any change in the
oracle's arithmetic.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle                                      # noqa: E402
from paper_2605_01313_gb300 import synth           # noqa: E402


def c1_points():
    """The 64 x 32 single-field workload: every 32nd of its 2048 rotated points."""
    wl = synth.workload_c1()
    s = np.arange(0, wl.lon.size, 32)
    return wl.coeffs, wl.lon[s], wl.colat[s], s


def tc2_points():
    """The tilted steady zonal flow (h, u, v) of Sec. 6 (alpha = pi/2 - 0.05) on the
    128 x 64 grid, at 32 seeded points anywhere on the doubled torus."""
    alpha = math.pi / 2 - 0.05
    c = np.stack(synth.zonal_flow_coeffs(128, 64, alpha))
    rng = np.random.default_rng(91)
    lon = rng.uniform(-1.0, 2 * math.pi + 1.0, 32)
    colat = rng.uniform(-math.pi, 2 * math.pi, 32)
    return c, lon, colat, np.arange(32)


FIXTURES = {
    "c1_oracle_values.txt": (c1_points, "64x32 grid, one field, |k|^-2 spectrum, points rotated "
                             "back by pi/144 about an axis tilted pi/4 (seed 1)"),
    "tc2_oracle_values.txt": (tc2_points, "tilted steady zonal flow h, u, v on 128x64, "
                              "alpha = pi/2 - 0.05, 32 seeded points (seed 91)"),
}


def write(name):
    make, what = FIXTURES[name]
    c, lon, colat, idx = make()
    v = oracle.evaluate(c, lon, colat)
    v = v.reshape(-1, lon.size)
    with open(os.path.join(HERE, name), "w") as fh:
        fh.write("# Eq. 5.3 (Sec. 5) evaluated by the FP64 oracle: %s\n" % what)
        fh.write("# written by tests/golden/make_golden.py; columns: point index, lon, colat, "
                 "then Re and Im of each field\n")
        for p in range(lon.size):
            cols = ["%d" % idx[p], repr(float(lon[p])), repr(float(colat[p]))]
            for f in range(v.shape[0]):
                cols += [repr(float(v[f, p].real)), repr(float(v[f, p].imag))]
            fh.write(" ".join(cols) + "\n")


if __name__ == "__main__":
    for name in FIXTURES:
        write(name)
        print("wrote", name)
