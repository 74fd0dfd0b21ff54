"""Oracle for the departure-point solve and the vector rotation of the
semi-Lagrangian step (Sec. 2).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library path never does, and
it shares no code with the CUDA path.  Plain FP64 NumPy, vectorised over
points only.

Conventions: Grid [0] arrival points (Sec. 3), colatitude theta_j =
(j + 1/2) pi / n_lat, longitude phi_k = 2 pi k / n_lon, flattened with the
longitude fastest.  Vector fields are given by their eastward and northward
components, shape (2, n_lat, n_lon).

* :func:`lagrange5_weights` -- quintic Lagrange weights on the equispaced nodes
  -2..3 (the interpolation the paper uses for the departure-point bracket,
  Sec. 2), from the product formula.
* :func:`interp_quintic` -- tensor-product quintic Lagrange interpolation of
  grid samples at arbitrary points; stencil rows beyond a pole come from the
  doubled sphere, f(phi + pi, -theta) = parity * f(phi, theta) (Sec. 4), with
  parity -1 for wind components.
* :func:`rotation_pq` -- p and q of the matrix Q of Sec. 2 as printed, with
  eta from the dot product of the two unit position vectors.
* :func:`rotate_to_arrival` -- Q applied to (u, v) given at the departure points.
* :func:`move_back` -- the departure point x - dt V of Eq. 2.4 on the sphere:
  the point reached from the arrival point along the great circle whose
  direction there is -V, after the angle |V| dt / a.
* :func:`departure_points` -- Eq. 2.4 solved by fixed-point iteration: start at
  the arrival point, interpolate the bracket's departure term there, carry it to
  the arrival frame by Q, subtract the arrival term, move back; repeat.
"""
from __future__ import annotations

import math

import numpy as np

NODES = np.arange(-2, 4, dtype=np.float64)      # stencil offsets of the six nodes


def lagrange5_weights(t: np.ndarray) -> np.ndarray:
    """Weights L_k(t), k = -2..3, of the degree-5 Lagrange interpolant through
    the nodes -2..3 evaluated at t (any shape); result shape t.shape + (6,)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty(t.shape + (6,))
    for a, xa in enumerate(NODES):
        num = np.ones_like(t)
        den = 1.0
        for xb in NODES:
            if xb != xa:
                num = num * (t - xb)
                den *= (xa - xb)
        out[..., a] = num / den
    return out


def _grid_value(field, parity, rows, cols):
    """Samples of the doubled sphere at integer row / column indices: rows
    outside [0, n_lat) are the mirrored rows half a turn away, times parity."""
    n_lat, n_lon = field.shape
    below = rows < 0
    above = rows >= n_lat
    r = np.where(below, -1 - rows, np.where(above, 2 * n_lat - 1 - rows, rows))
    shift = np.where(below | above, n_lon // 2, 0)
    c = np.mod(cols + shift, n_lon)
    sign = np.where(below | above, float(parity), 1.0)
    return sign * field[r, c]


def interp_quintic(field: np.ndarray, parity: int, lon: np.ndarray,
                   colat: np.ndarray) -> np.ndarray:
    """Quintic Lagrange interpolation of Grid [0] samples ``field`` (n_lat, n_lon)
    at the points (lon, colat), colat in [0, pi]."""
    n_lat, n_lon = field.shape
    if n_lon % 2 or n_lon < 6 or n_lat < 3:
        raise ValueError("need an even n_lon >= 6 and n_lat >= 3")
    x = np.mod(np.asarray(lon, dtype=np.float64) * (n_lon / (2.0 * math.pi)), n_lon)
    y = np.asarray(colat, dtype=np.float64) * (n_lat / math.pi) - 0.5
    i = np.floor(x)
    j = np.floor(y)
    wx = lagrange5_weights(x - i)
    wy = lagrange5_weights(y - j)
    i = i.astype(np.int64)
    j = j.astype(np.int64)
    total = np.zeros_like(x)
    for a in range(6):
        row = np.zeros_like(x)
        for b in range(6):
            row += wx[:, b] * _grid_value(field, parity, j + a - 2, i + b - 2)
        total += wy[:, a] * row
    return total


def _xyz(lon, colat):
    s = np.sin(colat)
    return np.stack([s * np.cos(lon), s * np.sin(lon), np.cos(colat)], axis=-1)


def rotation_pq(lon_a, colat_a, lon_d, colat_d):
    """p and q of Q (Sec. 2) for arrival A and departure D, longitude phi and
    colatitude theta:
      p = (sin th_A sin th_D + (1 + cos th_A cos th_D) cos(ph_A - ph_D)) / (1 + cos eta)
      q = (cos th_A + cos th_D) sin(ph_A - ph_D) / (1 + cos eta)
    with cos eta = r_A . r_D."""
    cos_eta = np.sum(_xyz(lon_a, colat_a) * _xyz(lon_d, colat_d), axis=-1)
    den = 1.0 + cos_eta
    dl = lon_a - lon_d
    p = (np.sin(colat_a) * np.sin(colat_d)
         + (1.0 + np.cos(colat_a) * np.cos(colat_d)) * np.cos(dl)) / den
    q = (np.cos(colat_a) + np.cos(colat_d)) * np.sin(dl) / den
    return p, q


def rotate_to_arrival(u_d, v_d, lon_a, colat_a, lon_d, colat_d):
    """(u, v) given at the departure points in the local frame there, expressed
    in the arrival points' local frame: Q = [[p, q], [-q, p]] (Sec. 2)."""
    p, q = rotation_pq(lon_a, colat_a, lon_d, colat_d)
    return p * u_d + q * v_d, -q * u_d + p * v_d


def move_back(lon_a, colat_a, s_east, s_north):
    """The point reached from A = (lon_a, colat_a) by the angle d = |s| along the
    great circle leaving A in the direction -s, s = (s_east, s_north) in A's
    local frame (radians).  Returns lon in [0, 2 pi), colat in [0, pi]."""
    lon_a = np.asarray(lon_a, dtype=np.float64)
    colat_a = np.asarray(colat_a, dtype=np.float64)
    r = _xyz(lon_a, colat_a)
    east = np.stack([-np.sin(lon_a), np.cos(lon_a), np.zeros_like(lon_a)], axis=-1)
    north = np.stack([-np.cos(colat_a) * np.cos(lon_a), -np.cos(colat_a) * np.sin(lon_a),
                      np.sin(colat_a)], axis=-1)
    d = np.hypot(s_east, s_north)
    safe = np.where(d > 0, d, 1.0)
    t = -(s_east / safe)[:, None] * east - (s_north / safe)[:, None] * north
    rd = np.cos(d)[:, None] * r + np.sin(d)[:, None] * t
    lon = np.mod(np.arctan2(rd[:, 1], rd[:, 0]), 2.0 * math.pi)
    lon = np.where(lon >= 2.0 * math.pi, 0.0, lon)
    colat = np.arctan2(np.hypot(rd[:, 0], rd[:, 1]), rd[:, 2])
    return lon, colat


def arrival_points(n_lon: int, n_lat: int):
    """Grid [0] arrival points, longitude fastest."""
    colat = (np.arange(n_lat) + 0.5) * (math.pi / n_lat)
    lon = np.arange(n_lon) * (2.0 * math.pi / n_lon)
    cc, ll = np.meshgrid(colat, lon, indexing="ij")
    return ll.ravel(), cc.ravel()


def departure_points(w: np.ndarray, a_term, dt_over_a: float, iterations: int,
                     index=None):
    """Departure points of Eq. 2.4 for every arrival point of Grid [0] (or the
    flat indices ``index`` of a subset), by ``iterations`` fixed-point steps.

    w: (2, n_lat, n_lon) east/north components of the bracket's departure term,
    (v + Omega x r - g dt grad h^(+) / 4) in the paper, interpolated at D;
    a_term: same shape, the arrival term (Omega x r + g dt grad h^0 / 4), or
    None for zero; dt_over_a: time step over the sphere's radius (s/m).
    Iteration k: V = Q(A, D_k) w(D_k) - a_term(A); D_{k+1} = move_back(A, V dt/a),
    with D_0 = A.  Returns (lon_D, colat_D)."""
    _, n_lat, n_lon = w.shape
    lon_a, colat_a = arrival_points(n_lon, n_lat)
    a_e = np.zeros(n_lat * n_lon) if a_term is None else a_term.reshape(2, -1)[0]
    a_n = np.zeros(n_lat * n_lon) if a_term is None else a_term.reshape(2, -1)[1]
    if index is not None:
        lon_a, colat_a = lon_a[index], colat_a[index]
        a_e, a_n = a_e[index], a_n[index]
    lon_d, colat_d = lon_a.copy(), colat_a.copy()
    for _ in range(iterations):
        we = interp_quintic(w[0], -1, lon_d, colat_d)
        wn = interp_quintic(w[1], -1, lon_d, colat_d)
        ue, un = rotate_to_arrival(we, wn, lon_a, colat_a, lon_d, colat_d)
        lon_d, colat_d = move_back(lon_a, colat_a, dt_over_a * (ue - a_e),
                                   dt_over_a * (un - a_n))
    return lon_d, colat_d
