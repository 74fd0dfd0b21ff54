"""Pins of the departure-point oracle (Sec. 2, Eq. 2.4 and the rotation Q)
against facts fixed by the mathematics, not by the oracle itself:
polynomial reproduction of the Lagrange weights, sixth-order convergence of
the interpolation across the poles, Q against a rigid rotation built by scipy,
the great-circle move against scipy's rotation vectors, and the fixed point of
Eq. 2.4 against an independent Newton solve with the exact (not interpolated)
bracket."""
import math

import numpy as np
import pytest

from oracle import departure as dep

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def xyz(lon, colat):
    s = np.sin(colat)
    return np.stack([s * np.cos(lon), s * np.sin(lon), np.cos(colat)], axis=-1)


def frame(lon, colat):
    east = np.stack([-np.sin(lon), np.cos(lon), np.zeros_like(lon)], axis=-1)
    north = np.stack([-np.cos(colat) * np.cos(lon), -np.cos(colat) * np.sin(lon),
                      np.sin(colat)], axis=-1)
    return east, north


def tangent_field(vec3, lon, colat):
    """East/north components of the projection of a fixed 3-D vector: a smooth
    tangent field on the sphere."""
    e, n = frame(lon, colat)
    return e @ vec3, n @ vec3


def rigid_rotation_field(axis, omega, lon, colat):
    """East/north components of the solid-body velocity omega axis x r (unit sphere)."""
    v = omega * np.cross(axis, xyz(lon, colat))
    e, n = frame(lon, colat)
    return np.sum(v * e, axis=-1), np.sum(v * n, axis=-1)


def grid_field(fun, n_lon, n_lat):
    lon, colat = dep.arrival_points(n_lon, n_lat)
    u, v = fun(lon, colat)
    return np.stack([u.reshape(n_lat, n_lon), v.reshape(n_lat, n_lon)])


# ------------------------------------------------------------------ Lagrange weights

def test_lagrange_weights_reproduce_degree_five_only():
    t = np.linspace(0.0, 1.0, 17)
    w = dep.lagrange5_weights(t)
    for p in range(6):
        assert np.max(np.abs(w @ dep.NODES ** p - t ** p)) < 1e-12
    assert np.max(np.abs(w @ dep.NODES ** 6 - t ** 6)) > 1.0     # not degree 6
    assert np.allclose(dep.lagrange5_weights(np.array([0.0]))[0], [0, 0, 1, 0, 0, 0])


def test_interp_exact_on_tensor_quintics_inside_the_grid():
    n_lon, n_lat = 40, 20
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(6), rng.standard_normal(6)
    r = np.arange(n_lat)[:, None]
    c = np.arange(n_lon)[None, :]
    field = np.polyval(a, r / n_lat) * np.polyval(b, c / n_lon)
    # points whose stencil stays inside the rows and away from the seam
    x = rng.uniform(3.0, n_lon - 4.0, 300)
    y = rng.uniform(3.0, n_lat - 4.0, 300)
    lon = x * 2 * math.pi / n_lon
    colat = (y + 0.5) * math.pi / n_lat
    got = dep.interp_quintic(field, 1, lon, colat)
    exact = np.polyval(a, y / n_lat) * np.polyval(b, x / n_lon)
    assert np.max(np.abs(got - exact)) < 1e-12 * np.max(np.abs(field))


def test_interp_sixth_order_across_the_poles_and_parity():
    """A smooth tangent field interpolated near both poles: the error falls by
    about 2^6 when the grid is refined; the scalar parity (a plausible mistake)
    leaves an O(1) error there."""
    vec = np.array([0.3, -1.1, 0.7])
    rng = np.random.default_rng(2)
    lon = rng.uniform(0, 2 * math.pi, 400)
    colat = np.concatenate([rng.uniform(0, 0.3, 200), rng.uniform(math.pi - 0.3, math.pi, 200)])
    ue, un = tangent_field(vec, lon, colat)
    errs = []
    for n_lat in (16, 32):
        g = grid_field(lambda lo, co: tangent_field(vec, lo, co), 2 * n_lat, n_lat)
        eu = np.max(np.abs(dep.interp_quintic(g[0], -1, lon, colat) - ue))
        ev = np.max(np.abs(dep.interp_quintic(g[1], -1, lon, colat) - un))
        errs.append(max(eu, ev))
    assert errs[1] < 1e-6
    assert 40 < errs[0] / errs[1] < 100, errs
    g = grid_field(lambda lo, co: tangent_field(vec, lo, co), 64, 32)
    wrong = dep.interp_quintic(g[1], +1, lon, colat) - un
    assert np.max(np.abs(wrong)) > 0.1


# ------------------------------------------------------------------ rotation Q

def test_q_is_the_rigid_rotation_carrying_d_to_a():
    rng = np.random.default_rng(3)
    n = 500
    lon_a = rng.uniform(0, 2 * math.pi, n)
    colat_a = rng.uniform(0.01, math.pi - 0.01, n)
    # departure points within 0.4 rad, some across a pole
    lon_d, colat_d = dep.move_back(lon_a, colat_a, rng.uniform(-0.4, 0.4, n),
                                   rng.uniform(-0.4, 0.4, n))
    ra, rd = xyz(lon_a, colat_a), xyz(lon_d, colat_d)
    axis = np.cross(rd, ra)
    angle = np.arctan2(np.linalg.norm(axis, axis=1), np.sum(ra * rd, axis=1))
    unit = axis / np.linalg.norm(axis, axis=1)[:, None]
    rot = Rotation.from_rotvec(unit * angle[:, None])
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    ed, nd = frame(lon_d, colat_d)
    ea, na = frame(lon_a, colat_a)
    carried = rot.apply(u[:, None] * ed + v[:, None] * nd)
    ua, va = dep.rotate_to_arrival(u, v, lon_a, colat_a, lon_d, colat_d)
    assert np.max(np.abs(ua - np.sum(carried * ea, axis=1))) < 1e-12
    assert np.max(np.abs(va - np.sum(carried * na, axis=1))) < 1e-12
    p, q = dep.rotation_pq(lon_a, colat_a, lon_d, colat_d)
    assert np.max(np.abs(p * p + q * q - 1.0)) < 1e-12
    p0, q0 = dep.rotation_pq(lon_a, colat_a, lon_a, colat_a)
    assert np.allclose(p0, 1.0) and np.allclose(q0, 0.0)


def test_q_transposed_is_caught():
    lon_a, colat_a = np.array([0.3]), np.array([0.4])
    lon_d, colat_d = dep.move_back(lon_a, colat_a, np.array([0.2]), np.array([0.1]))
    p, q = dep.rotation_pq(lon_a, colat_a, lon_d, colat_d)
    assert abs(q[0]) > 0.05       # the two orientations differ by 2q


# ------------------------------------------------------------------ great-circle move

def test_move_back_is_a_rotation_about_r_cross_direction():
    rng = np.random.default_rng(4)
    n = 500
    lon_a = rng.uniform(0, 2 * math.pi, n)
    colat_a = rng.uniform(0.02, math.pi - 0.02, n)
    se, sn = rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n)
    lon_d, colat_d = dep.move_back(lon_a, colat_a, se, sn)
    ra = xyz(lon_a, colat_a)
    e, nvec = frame(lon_a, colat_a)
    direction = -(se[:, None] * e + sn[:, None] * nvec)
    d = np.hypot(se, sn)
    axis = np.cross(ra, direction / d[:, None])
    expect = Rotation.from_rotvec(axis * d[:, None]).apply(ra)
    assert np.max(np.abs(xyz(lon_d, colat_d) - expect)) < 1e-13
    # haversine distance = |s|
    dlat = (math.pi / 2 - colat_d) - (math.pi / 2 - colat_a)
    hav = (np.sin(dlat / 2) ** 2 + np.sin(colat_a) * np.sin(colat_d)
           * np.sin((lon_d - lon_a) / 2) ** 2)
    assert np.max(np.abs(2 * np.arcsin(np.sqrt(hav)) - d)) < 1e-12
    assert np.all((lon_d >= 0) & (lon_d < 2 * math.pi))
    assert np.all((colat_d >= 0) & (colat_d <= math.pi))


# ------------------------------------------------------------------ Eq. 2.4

def newton_fixed_point(w_exact, a_e, a_n, dt_over_a, lon_a, colat_a):
    """Solve r_D = exp_A(-dt/a (Q w(D) - a)) for one point by Newton's method
    on the unit vector r_D (finite-difference Jacobian), with Q built as the
    rigid rotation carrying D to A (scipy) and w evaluated exactly."""
    ra = xyz(np.array([lon_a]), np.array([colat_a]))[0]
    e, nvec = (x[0] for x in frame(np.array([lon_a]), np.array([colat_a])))

    def image(rd):
        rd = rd / np.linalg.norm(rd)
        lon_d = math.atan2(rd[1], rd[0])
        colat_d = math.atan2(math.hypot(rd[0], rd[1]), rd[2])
        we, wn = w_exact(np.array([lon_d]), np.array([colat_d]))
        ed, nd = (x[0] for x in frame(np.array([lon_d]), np.array([colat_d])))
        vec = we[0] * ed + wn[0] * nd
        axis = np.cross(rd, ra)
        s = np.linalg.norm(axis)
        if s > 0:
            vec = Rotation.from_rotvec(axis / s * math.atan2(s, rd @ ra)).apply(vec)
        ve, vn = vec @ e - a_e, vec @ nvec - a_n
        step = -dt_over_a * (ve * e + vn * nvec)
        d = np.linalg.norm(step)
        if d == 0:
            return ra.copy()
        return math.cos(d) * ra + math.sin(d) * step / d

    x = ra.copy()
    for _ in range(40):
        f = image(x) - x
        jac = np.empty((3, 3))
        for k in range(3):
            h = np.zeros(3)
            h[k] = 1e-7
            jac[:, k] = ((image(x + h) - (x + h)) - f) / 1e-7
        x = x - np.linalg.lstsq(jac, f, rcond=None)[0]
        x /= np.linalg.norm(x)
    lon_d = math.atan2(x[1], x[0]) % (2 * math.pi)
    return lon_d, math.atan2(math.hypot(x[0], x[1]), x[2])


@pytest.mark.parametrize("mistake", [None, "q_transposed", "plus_a", "forward"])
def test_fixed_point_matches_an_independent_newton_solve(mistake):
    """A rigid rotation about a tilted axis plus a constant arrival term: the
    oracle's iterate after 40 steps agrees with Newton's solution of Eq. 2.4
    built from scipy rotations and the exact field, to the quintic
    interpolation error; each planted mistake misses it."""
    n_lon, n_lat = 128, 64
    axis = np.array([math.sin(0.7) * math.cos(0.3), math.sin(0.7) * math.sin(0.3), math.cos(0.7)])
    omega = 40.0                                 # m/s at unit distance from the axis
    dt_over_a = 2400.0 / 6.371e6
    w_exact = lambda lo, co: rigid_rotation_field(axis, omega, lo, co)
    w = grid_field(w_exact, n_lon, n_lat)
    a_term = np.zeros_like(w)
    a_term[0] += 3.0
    a_term[1] -= 2.0
    index = np.array([0, 77, 2000, 4100, 5000, 8000, n_lon * n_lat - 1])
    if mistake is None:
        lon_d, colat_d = dep.departure_points(w, a_term, dt_over_a, 40, index=index)
    else:
        lon_a, colat_a = dep.arrival_points(n_lon, n_lat)
        lon_a, colat_a = lon_a[index], colat_a[index]
        lon_d, colat_d = lon_a.copy(), colat_a.copy()
        for _ in range(40):
            we = dep.interp_quintic(w[0], -1, lon_d, colat_d)
            wn = dep.interp_quintic(w[1], -1, lon_d, colat_d)
            p, q = dep.rotation_pq(lon_a, colat_a, lon_d, colat_d)
            if mistake == "q_transposed":
                ue, un = p * we - q * wn, q * we + p * wn
            else:
                ue, un = p * we + q * wn, -q * we + p * wn
            sgn = 1.0 if mistake == "plus_a" else -1.0
            fwd = -1.0 if mistake == "forward" else 1.0
            lon_d, colat_d = dep.move_back(lon_a, colat_a, fwd * dt_over_a * (ue + sgn * 3.0),
                                           fwd * dt_over_a * (un - sgn * 2.0))
    lon_a, colat_a = dep.arrival_points(n_lon, n_lat)
    err = []
    for k, i in enumerate(index):
        ln, cn = newton_fixed_point(w_exact, 3.0, -2.0, dt_over_a, lon_a[i], colat_a[i])
        gap = np.linalg.norm(xyz(np.array([ln]), np.array([cn]))[0]
                             - xyz(np.array([lon_d[k]]), np.array([colat_d[k]]))[0])
        err.append(gap)
    if mistake is None:
        assert max(err) < 1e-10, err
    else:
        assert max(err) > 1e-6, err
