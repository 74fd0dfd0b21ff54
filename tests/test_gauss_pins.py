"""Pins of the Gauss-Legendre-grid oracle (oracle/gauss.py): on Grid [0] rows it
is the plain Fourier sum of oracle.grid_to_coeffs; on Gauss-Legendre rows it
recovers band-limited DFS fields exactly and its series passes through every
sample; the nodes integrate polynomials of degree 2 n_lat - 1 exactly."""
import math

import numpy as np
import pytest

import oracle
from oracle import gauss
from paper_2605_01313_gb300 import synth


def test_nodes_are_a_gauss_rule():
    n_lat = 12
    th = gauss.gauss_legendre_colat(n_lat)
    assert np.all(np.diff(th) > 0) and th[0] > 0 and th[-1] < math.pi
    z = np.cos(th)
    # weights from the nodes alone: sum_j w_j P_k(z_j) = 2 delta_k0 for k < n
    A = np.stack([np.polynomial.legendre.legval(z, np.eye(n_lat)[k]) for k in range(n_lat)])
    w = np.linalg.solve(A, np.eye(n_lat)[0] * 2.0)
    for d in range(2 * n_lat):
        exact = (1 - (-1) ** (d + 1)) / (d + 1)
        assert abs(np.sum(w * z ** d) - exact) < 1e-12, d


def test_grid0_rows_reduce_to_the_fourier_sum():
    rng = np.random.default_rng(40)
    n_lon, n_lat = 16, 8
    s = rng.standard_normal((2, n_lat, n_lon))
    colat = (np.arange(n_lat) + 0.5) * math.pi / n_lat
    a = gauss.gl_to_coeffs(s, [1, -1], colat)
    b = oracle.grid_to_coeffs(s, [1, -1])
    assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("n_lon,n_lat", [(16, 8), (32, 16), (24, 11)])
def test_recovers_band_limited_fields_on_gauss_rows(n_lon, n_lat):
    rng = np.random.default_rng(41 + n_lat)
    colat = gauss.gauss_legendre_colat(n_lat)
    c = np.stack([synth.random_spectrum(rng, n_lon, n_lat, 1.5, par)
                  for par in (synth.SCALAR, synth.VECTOR)])
    cc, ll = np.meshgrid(colat, np.arange(n_lon) * 2 * math.pi / n_lon, indexing="ij")
    vals = oracle.evaluate(c, ll.ravel(), cc.ravel()).real.reshape(2, n_lat, n_lon)
    got = gauss.gl_to_coeffs(vals, [1, -1], colat)
    assert np.max(np.abs(got - c)) < 1e-11 * np.max(np.abs(c))


def test_series_passes_through_the_samples_and_parity_split():
    """Arbitrary samples: the series reproduces them; in the longitude modes
    whose doubled column is even (parity (-1)^m = +1) the Nyquist row vanishes."""
    rng = np.random.default_rng(42)
    n_lon, n_lat = 16, 7
    colat = gauss.gauss_legendre_colat(n_lat)
    s = rng.standard_normal((2, n_lat, n_lon))
    c = gauss.gl_to_coeffs(s, [1, -1], colat)
    cc, ll = np.meshgrid(colat, np.arange(n_lon) * 2 * math.pi / n_lon, indexing="ij")
    back = oracle.evaluate(c, ll.ravel(), cc.ravel()).real.reshape(2, n_lat, n_lon)
    assert np.max(np.abs(back - s)) < 1e-11
    m = np.arange(n_lon) - n_lon // 2
    for f, par in enumerate((1, -1)):
        even = par * (-1.0) ** m > 0
        assert np.max(np.abs(c[f, 0, even])) < 1e-12
        assert np.max(np.abs(c[f, 0, ~even])) > 1e-6
