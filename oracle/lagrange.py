"""Oracle for the Lagrange interpolation comparator: the tensor-product cubic and
quintic Lagrange interpolation the paper's baseline model uses at departure
points (cubic for the scalar forcing, quintic for the vector one; Sec. 1-2).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library path never does, and
it shares no code with the CUDA path.  Plain FP64 NumPy.

Samples are given on Grid [0] (Sec. 3), shape (n_lat, n_lon).  A point's
colatitude is reduced to [-pi, pi) and a negative one taken as the point
(phi + pi, -theta) of the doubled sphere, where the field is parity times its
value (Sec. 4; parity -1 for wind components), so any real (lon, colat) is
accepted; stencil rows beyond a pole come from the same extension.
"""
from __future__ import annotations

import math

import numpy as np

from .departure import _grid_value


def nodes(order: int) -> np.ndarray:
    """Stencil offsets of the order + 1 equispaced nodes around [0, 1):
    -1..2 for cubic, -2..3 for quintic."""
    if order not in (3, 5):
        raise ValueError("order must be 3 or 5")
    h = (order - 1) // 2
    return np.arange(-h, order - h + 1, dtype=np.float64)


def lagrange_weights(t: np.ndarray, order: int) -> np.ndarray:
    """Weights of the degree-``order`` Lagrange interpolant through nodes(order)
    at t, from the product formula; shape t.shape + (order + 1,)."""
    x = nodes(order)
    t = np.asarray(t, dtype=np.float64)
    out = np.empty(t.shape + (x.size,))
    for a, xa in enumerate(x):
        num = np.ones_like(t)
        den = 1.0
        for xb in x:
            if xb != xa:
                num = num * (t - xb)
                den *= xa - xb
        out[..., a] = num / den
    return out


def interp_lagrange(field: np.ndarray, parity: int, lon, colat, order: int) -> np.ndarray:
    """Tensor-product Lagrange interpolation of degree ``order`` (3 or 5) of the
    Grid [0] samples ``field`` at the points (lon, colat)."""
    n_lat, n_lon = field.shape
    if n_lon % 2 or n_lon < order + 1 or n_lat < (order + 1) // 2:
        raise ValueError("grid too small for this order")
    lon = np.asarray(lon, dtype=np.float64)
    th = np.asarray(colat, dtype=np.float64)
    th = th - 2.0 * math.pi * np.floor((th + math.pi) / (2.0 * math.pi))     # [-pi, pi)
    neg = th < 0
    th = np.where(neg, -th, th)
    lon = np.where(neg, lon + math.pi, lon)
    sign = np.where(neg, float(parity), 1.0)
    x = np.mod(lon * (n_lon / (2.0 * math.pi)), n_lon)
    y = th * (n_lat / math.pi) - 0.5
    i = np.floor(x)
    j = np.floor(y)
    wx = lagrange_weights(x - i, order)
    wy = lagrange_weights(y - j, order)
    i = i.astype(np.int64)
    j = j.astype(np.int64)
    off = nodes(order).astype(np.int64)
    total = np.zeros_like(x)
    for a, da in enumerate(off):
        row = np.zeros_like(x)
        for b, db in enumerate(off):
            row += wx[:, b] * _grid_value(field, parity, j + da, i + db)
        total += wy[:, a] * row
    return sign * total
