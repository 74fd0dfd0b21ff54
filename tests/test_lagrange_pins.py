"""Pins of the Lagrange comparator's oracle (oracle/lagrange.py): polynomial
reproduction of the weights, the quintic form equal to the departure oracle's,
the convergence order across the poles, and the doubled-sphere reduction of any
real coordinate."""
import math

import numpy as np
import pytest

from oracle import departure as dep
from oracle import lagrange as lag


@pytest.mark.parametrize("order", [3, 5])
def test_weights_reproduce_degree_order_only(order):
    t = np.linspace(0.0, 1.0, 13)
    w = lag.lagrange_weights(t, order)
    x = lag.nodes(order)
    for p in range(order + 1):
        assert np.max(np.abs(w @ x ** p - t ** p)) < 1e-12
    assert np.max(np.abs(w @ x ** (order + 1) - t ** (order + 1))) > 0.05
    assert np.allclose(np.sum(w, axis=-1), 1.0)


def test_quintic_equals_departure_oracle():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((16, 32))
    lon = rng.uniform(0, 2 * math.pi, 300)
    colat = rng.uniform(0, math.pi, 300)
    for par in (1, -1):
        a = lag.interp_lagrange(f, par, lon, colat, 5)
        b = dep.interp_quintic(f, par, lon, colat)
        assert np.max(np.abs(a - b)) < 1e-13


def smooth(lon, colat):
    """A smooth scalar on the sphere: a fixed quadratic in Cartesian coordinates."""
    x, y, z = np.sin(colat) * np.cos(lon), np.sin(colat) * np.sin(lon), np.cos(colat)
    return 0.3 + x - 0.7 * y * z + 1.3 * x * z + 0.4 * z * z


@pytest.mark.parametrize("order,expect", [(3, 16.0), (5, 64.0)])
def test_convergence_order_across_poles(order, expect):
    rng = np.random.default_rng(6)
    lon = rng.uniform(0, 2 * math.pi, 400)
    colat = np.concatenate([rng.uniform(0, 0.25, 200), rng.uniform(math.pi - 0.25, math.pi, 200)])
    errs = []
    for n_lat in (16, 32):
        la, ca = dep.arrival_points(2 * n_lat, n_lat)
        f = smooth(la, ca).reshape(n_lat, 2 * n_lat)
        errs.append(np.max(np.abs(lag.interp_lagrange(f, 1, lon, colat, order)
                                  - smooth(lon, colat))))
    ratio = errs[0] / errs[1]
    assert 0.6 * expect < ratio < 1.6 * expect, (errs, ratio)


def test_any_real_coordinate_by_the_doubled_sphere():
    rng = np.random.default_rng(7)
    f = rng.standard_normal((12, 24))
    lon = rng.uniform(0, 2 * math.pi, 200)
    colat = rng.uniform(0.01, math.pi - 0.01, 200)
    for par in (1, -1):
        base = lag.interp_lagrange(f, par, lon, colat, 3)
        # the same physical point written on the other half of the doubled torus
        other = lag.interp_lagrange(f, par, lon + math.pi, -colat, 3)
        assert np.max(np.abs(other - par * base)) < 1e-12
        # whole turns in both coordinates
        turned = lag.interp_lagrange(f, par, lon - 4 * math.pi, colat + 2 * math.pi, 3)
        assert np.max(np.abs(turned - base)) < 1e-12
