"""Seeded synthetic inputs for the DFS spectral-interpolation step.

This module only *draws* inputs: DFS coefficient arrays on the doubled torus and
departure points on the sphere, shaped like the paper's shallow-water test cases
(Sec. 6: Williamson TC1/TC2-style solid-body and zonal geostrophic flows).  It
holds none of the interpolation method's arithmetic (no series evaluation, no
NUFFT step): both the CUDA path and the CPU oracle consume what it returns.

Conventions shared by every array produced here
-----------------------------------------------
* Grid: Grid [0] of Sec. 3, colatitude theta_j = (j + 1/2) pi / J for
  j = 0..J-1 (n_lat = J) and longitude phi_i = 2 pi i / n_lon (n_lon = 2J).
* Coefficient array ``c`` of one field: shape (N2, N1) = (2 n_lat, n_lon),
  C-contiguous, complex.  Row r holds theta-wavenumber n = r - N2/2, column q
  holds phi-wavenumber m = q - N1/2, so that the field is
  f(phi, theta) = sum_{n,m} c[n + N2/2, m + N1/2] exp(i m phi) exp(i n theta)
  (Eq. 5.3).  The Nyquist row and column (n = -N2/2, m = -N1/2) are kept zero.
* Symmetries (Sec. 4): real fields have c_{-n,-m} = conj(c_{n,m}).  On the
  doubled sphere a scalar satisfies f(phi + pi, -theta) = f(phi, theta), i.e.
  c_{-n,m} = (-1)^m c_{n,m}; a wind component changes sign through the pole,
  c_{-n,m} = -(-1)^m c_{n,m}.
* Points: longitude in [0, 2 pi), colatitude in [0, pi], float64, one per
  arrival grid point in grid order (colatitude rows, longitude fastest).
"""
from __future__ import annotations

import math

import numpy as np

EARTH_RADIUS = 6.371e6          # m, the radius the workloads are stated with
EARTH_OMEGA = 7.292e-5          # 1/s
GRAVITY = 9.80616               # m/s^2
DAY = 86400.0                   # s
U0_12DAY = 2.0 * math.pi * EARTH_RADIUS / (12.0 * DAY)   # one revolution in 12 days

SCALAR = +1
VECTOR = -1


# --------------------------------------------------------------------------- grids

def coeff_shape(n_lon: int, n_lat: int) -> tuple[int, int]:
    """(N2, N1) = (2 n_lat, n_lon): theta-modes x phi-modes on the doubled torus."""
    return 2 * n_lat, n_lon


def wavenumbers(n_lon: int, n_lat: int) -> tuple[np.ndarray, np.ndarray]:
    """Centred wavenumber vectors (n for rows, m for columns)."""
    n2, n1 = coeff_shape(n_lon, n_lat)
    return np.arange(n2) - n2 // 2, np.arange(n1) - n1 // 2


def grid0_points(n_lon: int, n_lat: int) -> tuple[np.ndarray, np.ndarray]:
    """Arrival points of Grid [0] (Sec. 3), flattened in grid order."""
    j = np.arange(n_lat)
    colat = (j + 0.5) * math.pi / n_lat
    lon = 2.0 * math.pi * np.arange(n_lon) / n_lon
    cc, ll = np.meshgrid(colat, lon, indexing="ij")
    return ll.ravel().copy(), cc.ravel().copy()


def to_xyz(lon, colat):
    s = np.sin(colat)
    return np.stack([s * np.cos(lon), s * np.sin(lon), np.cos(colat)], axis=-1)


def from_xyz(xyz):
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    colat = np.arccos(np.clip(z / r, -1.0, 1.0))
    lon = np.mod(np.arctan2(y, x), 2.0 * math.pi)
    lon = np.where(lon >= 2.0 * math.pi, 0.0, lon)
    return lon, colat


def rotation_axis(alpha: float) -> np.ndarray:
    """Axis of a solid-body rotation tilted by ``alpha`` from the pole (TC1/TC2)."""
    return np.array([-math.sin(alpha), 0.0, math.cos(alpha)])


def rotate(xyz: np.ndarray, axis: np.ndarray, angle: float) -> np.ndarray:
    """Rodrigues rotation of row vectors ``xyz`` about unit ``axis`` by ``angle``."""
    k = np.asarray(axis, dtype=np.float64)
    c, s = math.cos(angle), math.sin(angle)
    kxv = np.cross(k, xyz)
    kdv = xyz @ k
    return xyz * c + kxv * s + np.outer(kdv, k) * (1.0 - c)


def solid_body_departure(lon, colat, alpha: float, u0: float, dt: float,
                         radius: float = EARTH_RADIUS):
    """Departure points of a solid-body rotation: the arrival points rotated back
    by the angle u0 dt / a about the tilted axis."""
    xyz = to_xyz(lon, colat)
    dep = rotate(xyz, rotation_axis(alpha), -u0 * dt / radius)
    return from_xyz(dep)


def divergent_departure(rng: np.random.Generator, lon, colat, vmax: float, dt: float,
                        degree: int = 4, radius: float = EARTH_RADIUS):
    """Departure points displaced by a seeded divergent wind v = grad_s F.

    F is a random polynomial of the given degree in Cartesian (x, y, z); its
    tangential gradient is scaled so that max |v| over the points is ``vmax``
    and each point moves back along its great circle by |v| dt.
    """
    xyz = to_xyz(lon, colat)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    grad = np.zeros_like(xyz)
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            for k in range(degree + 1 - i - j):
                if i + j + k == 0:
                    continue
                a = rng.standard_normal() / (i + j + k)
                if i:
                    grad[:, 0] += a * i * x ** (i - 1) * y ** j * z ** k
                if j:
                    grad[:, 1] += a * j * x ** i * y ** (j - 1) * z ** k
                if k:
                    grad[:, 2] += a * k * x ** i * y ** j * z ** (k - 1)
    tang = grad - np.sum(grad * xyz, axis=1, keepdims=True) * xyz
    speed = np.linalg.norm(tang, axis=1)
    vel = tang * (vmax / speed.max())
    spd = np.linalg.norm(vel, axis=1)
    safe = np.where(spd > 0, spd, 1.0)
    that = vel / safe[:, None]
    d = spd * dt / radius
    dep = np.cos(d)[:, None] * xyz - np.sin(d)[:, None] * that
    return from_xyz(dep)


# --------------------------------------------------------------------------- spectra

def symmetrize(c: np.ndarray, parity: int) -> np.ndarray:
    """Project a centred coefficient array onto real fields of the given DFS
    parity (+1 scalar, -1 wind component); the Nyquist row/column are zeroed."""
    c = np.array(c, dtype=np.complex128, copy=True)
    c[0, :] = 0.0
    c[:, 0] = 0.0
    n2, n1 = c.shape
    m = np.arange(n1) - n1 // 2
    sgn = parity * np.where(m % 2 == 0, 1.0, -1.0)          # parity * (-1)^m per column
    flip_n = c[::-1, :]
    flip_n = np.roll(flip_n, 1, axis=0)                     # row r -> row (N2 - r) mod N2
    flip_m = np.roll(c[:, ::-1], 1, axis=1)
    flip_nm = np.roll(np.roll(c[::-1, ::-1], 1, axis=0), 1, axis=1)
    herm = np.conj(flip_nm)                                 # conj c_{-n,-m}
    par = sgn[None, :] * flip_n                             # s (-1)^m c_{-n,m}
    both = sgn[None, :] * np.conj(flip_m)                   # s (-1)^m conj c_{n,-m}
    out = 0.25 * (c + herm + par + both)
    out[0, :] = 0.0
    out[:, 0] = 0.0
    return out


def random_spectrum(rng: np.random.Generator, n_lon: int, n_lat: int, decay: float,
                    parity: int = SCALAR) -> np.ndarray:
    """Complex Gaussian coefficients with amplitude |k|^-decay (|0| -> 1), made
    real and DFS-symmetric."""
    n2, n1 = coeff_shape(n_lon, n_lat)
    n, m = wavenumbers(n_lon, n_lat)
    kk = np.sqrt(n[:, None].astype(np.float64) ** 2 + m[None, :].astype(np.float64) ** 2)
    kk[kk == 0] = 1.0
    amp = kk ** (-decay)
    g = (rng.standard_normal((n2, n1)) + 1j * rng.standard_normal((n2, n1))) * amp
    return symmetrize(g, parity)


def coeff_norm(c: np.ndarray) -> float:
    """Root-mean-square of the field over the doubled torus (Parseval)."""
    return float(np.sqrt(np.sum(np.abs(c) ** 2)))


def torus_samples_to_coeffs(samples: np.ndarray) -> np.ndarray:
    """Coefficients of the trigonometric interpolant of samples taken on the
    doubled Grid [0] torus: rows theta_j = (j + 1/2) 2 pi / N2, columns
    phi_i = 2 pi i / N1.  Used only to draw inputs (a Gaussian bump)."""
    n2, n1 = samples.shape
    f = np.fft.fft2(samples) / (n1 * n2)
    f = np.fft.fftshift(f)
    n = np.arange(n2) - n2 // 2
    f *= np.exp(-1j * n * (math.pi / n2))[:, None]          # half-cell theta offset
    return f


def coeffs_to_grid_samples(c: np.ndarray, n_lon: int, n_lat: int) -> np.ndarray:
    """Real samples on Grid [0] (n_lat x n_lon) of the fields whose centred
    coefficients are c (F, N2, N1): the inverse of torus_samples_to_coeffs,
    rows j < n_lat of the doubled torus.  Used only to draw inputs (arrival-grid
    fields of a given spectrum)."""
    n2, n1 = c.shape[-2:]
    n = np.arange(n2) - n2 // 2
    f = c * np.exp(1j * n * (math.pi / n2))[:, None]
    f = np.fft.ifft2(np.fft.ifftshift(f, axes=(-2, -1))) * (n1 * n2)
    return np.ascontiguousarray(f[..., :n_lat, :].real)


def gaussian_bump_coeffs(n_lon: int, n_lat: int, center_lon: float, center_colat: float,
                         width: float, amplitude: float,
                         radius: float = EARTH_RADIUS) -> np.ndarray:
    """Coefficients of amplitude * exp(-(d / width)^2), d the great-circle
    distance to the centre, sampled on the doubled torus (scalar parity holds
    because the field is defined through Cartesian coordinates)."""
    n2, n1 = coeff_shape(n_lon, n_lat)
    th = (np.arange(n2) + 0.5) * (2.0 * math.pi / n2)
    ph = np.arange(n1) * (2.0 * math.pi / n1)
    c0 = to_xyz(np.array([center_lon]), np.array([center_colat]))[0]
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    dot = st * np.cos(ph)[None, :] * c0[0] + st * np.sin(ph)[None, :] * c0[1] + ct * c0[2]
    d = radius * np.arccos(np.clip(dot, -1.0, 1.0))
    vals = amplitude * np.exp(-(d / width) ** 2)
    return symmetrize(torus_samples_to_coeffs(vals), SCALAR)


# ----------------------------------------------- steady zonal geostrophic flow (TC2)
# Trigonometric polynomials are dicts {(n, m): coefficient of e^{i m phi} e^{i n theta}}.

def _tp_mul(a: dict, b: dict) -> dict:
    out: dict = {}
    for (n1, m1), x in a.items():
        for (n2, m2), y in b.items():
            key = (n1 + n2, m1 + m2)
            out[key] = out.get(key, 0.0) + x * y
    return out


def _tp_add(*terms) -> dict:
    out: dict = {}
    for scale, t in terms:
        for key, x in t.items():
            out[key] = out.get(key, 0.0) + scale * x
    return out


_ONE = {(0, 0): 1.0 + 0j}
_SIN_T = {(1, 0): -0.5j, (-1, 0): 0.5j}
_COS_T = {(1, 0): 0.5 + 0j, (-1, 0): 0.5 + 0j}
_SIN_P = {(0, 1): -0.5j, (0, -1): 0.5j}
_COS_P = {(0, 1): 0.5 + 0j, (0, -1): 0.5 + 0j}


def _tp_to_array(tp: dict, n_lon: int, n_lat: int) -> np.ndarray:
    n2, n1 = coeff_shape(n_lon, n_lat)
    c = np.zeros((n2, n1), dtype=np.complex128)
    for (n, m), x in tp.items():
        c[n + n2 // 2, m + n1 // 2] += x
    return c


def zonal_flow_constants(u0: float = U0_12DAY, radius: float = EARTH_RADIUS,
                         omega: float = EARTH_OMEGA, gravity: float = GRAVITY):
    """K in h = h0 - K s^2 for gradient-wind balance of solid-body zonal flow."""
    return (radius * omega * u0 + 0.5 * u0 * u0) / gravity


def zonal_flow_coeffs(n_lon: int, n_lat: int, alpha: float, u0: float = U0_12DAY,
                      h0: float = 2.94e4 / GRAVITY) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Exact DFS coefficients of the steady zonal geostrophic flow tilted by alpha.

    With s = k.r (k the tilted axis, r the unit position vector):
      u = u0 (cos a sin theta + sin a cos theta cos phi)   (eastward)
      v = -u0 sin a sin phi                                (northward)
      h = h0 - K s^2,  s = cos a cos theta - sin a sin theta cos phi
    All three are trigonometric polynomials with |n|, |m| <= 2.
    """
    ca, sa = math.cos(alpha), math.sin(alpha)
    K = zonal_flow_constants(u0)
    u = _tp_add((u0 * ca, _SIN_T), (u0 * sa, _tp_mul(_COS_T, _COS_P)))
    v = _tp_add((-u0 * sa, _SIN_P))
    s = _tp_add((ca, _COS_T), (-sa, _tp_mul(_SIN_T, _COS_P)))
    h = _tp_add((h0, _ONE), (-K, _tp_mul(s, s)))
    return (_tp_to_array(h, n_lon, n_lat), _tp_to_array(u, n_lon, n_lat),
            _tp_to_array(v, n_lon, n_lat))


def zonal_flow_values(lon, colat, alpha: float, u0: float = U0_12DAY,
                      h0: float = 2.94e4 / GRAVITY):
    """Pointwise h, u, v of the same flow, straight from the formulas."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    K = zonal_flow_constants(u0)
    u = u0 * (ca * np.sin(colat) + sa * np.cos(colat) * np.cos(lon))
    v = -u0 * sa * np.sin(lon)
    s = ca * np.cos(colat) - sa * np.sin(colat) * np.cos(lon)
    h = h0 - K * s * s
    return h, u, v


def zonal_flow_settls_terms(lon, colat, alpha: float, dt: float, u0: float = U0_12DAY,
                            radius: float = EARTH_RADIUS, omega: float = EARTH_OMEGA,
                            gravity: float = GRAVITY):
    """East/north components of the two terms of the departure-point equation
    (Sec. 2, Eq. 2.4) for the steady tilted zonal flow (so h^(+) = h^0):
      departure term  W   = v + Omega x r - g dt grad h / 4,
      arrival term    W_A = Omega x r + g dt grad h / 4,
    with Omega x r = Omega a sin(theta) (east) and, for h = h0 - K s^2,
    grad h = -(2 K s / a) (k . e_east, k . e_north)."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    K = zonal_flow_constants(u0, radius, omega, gravity)
    _, u, v = zonal_flow_values(lon, colat, alpha, u0)
    s = ca * np.cos(colat) - sa * np.sin(colat) * np.cos(lon)
    k_east = sa * np.sin(lon)
    k_north = sa * np.cos(colat) * np.cos(lon) + ca * np.sin(colat)
    gh_e = -(2.0 * K * s / radius) * k_east
    gh_n = -(2.0 * K * s / radius) * k_north
    rot = omega * radius * np.sin(colat)
    c = gravity * dt / 4.0
    w = np.stack([u + rot - c * gh_e, v - c * gh_n])
    wa = np.stack([rot + c * gh_e, c * gh_n])
    return w, wa


# --------------------------------------------------------------------------- workloads

class Workload:
    """One interpolation problem: coefficients (F, N2, N1) and P points."""

    def __init__(self, name, n_lon, n_lat, coeffs, lon, colat, tol, dtype, sample=None):
        self.name = name
        self.n_lon = n_lon
        self.n_lat = n_lat
        self.coeffs = coeffs          # complex128, (F, N2, N1)
        self.lon = lon                # float64, (P,)
        self.colat = colat
        self.tol = tol
        self.dtype = dtype            # "f64" or "f32"
        self.sample = sample          # indices checked against the oracle

    @property
    def n_fields(self):
        return self.coeffs.shape[0]

    @property
    def n_points(self):
        return self.lon.shape[0]


def workload_c1() -> Workload:
    """64x32 Grid [0], one field, |k|^-2 spectrum, solid-body rotation alpha = pi/4,
    dt = 3600 s; FP64 at tol 1e-12; every point checked."""
    rng = np.random.default_rng(1)
    n_lon, n_lat = 64, 32
    c = random_spectrum(rng, n_lon, n_lat, 2.0, SCALAR)[None]
    lon, colat = solid_body_departure(*grid0_points(n_lon, n_lat), math.pi / 4, U0_12DAY, 3600.0)
    return Workload("c1_64x32_f64", n_lon, n_lat, c, lon, colat, 1e-12, "f64",
                    sample=np.arange(lon.size))


def workload_c2(dtype: str = "f64", n_sample: int = 4096) -> Workload:
    """512x256, fields (h, u, v) = tilted steady zonal flow (alpha = pi/2 - 0.05, as in
    TC2) + 1% |k|^-3 noise of matching parity; departure points are the exact
    back-rotation over the dt that gives zonal Courant number 5."""
    rng = np.random.default_rng(2)
    n_lon, n_lat = 512, 256
    alpha = math.pi / 2 - 0.05
    fields = list(zonal_flow_coeffs(n_lon, n_lat, alpha))
    parities = (SCALAR, VECTOR, VECTOR)
    for i, par in enumerate(parities):
        noise = random_spectrum(rng, n_lon, n_lat, 3.0, par)
        noise *= 0.01 * coeff_norm(fields[i]) / coeff_norm(noise)
        fields[i] = fields[i] + noise
    dt = 5.0 * (2.0 * math.pi / n_lon) * EARTH_RADIUS / U0_12DAY
    lon, colat = solid_body_departure(*grid0_points(n_lon, n_lat), alpha, U0_12DAY, dt)
    sample = np.sort(rng.choice(lon.size, n_sample, replace=False))
    tol = 1e-12 if dtype == "f64" else 1e-6
    return Workload("c2_512x256_" + dtype, n_lon, n_lat, np.stack(fields), lon, colat,
                    tol, dtype, sample=sample)


def workload_c3(dtype: str = "f32", n_sample: int = 1000, n_lon: int = 2048,
                n_lat: int = 1024) -> Workload:
    """2048x1024, fields (h, u, v): |k|^-3 spectra (h also carries a 500 km Gaussian
    bump); departure points displaced by a seeded divergent wind of max 80 m/s
    over dt = 1800 s."""
    rng = np.random.default_rng(3)
    h = random_spectrum(rng, n_lon, n_lat, 3.0, SCALAR)
    h *= 100.0 / coeff_norm(h)
    h += gaussian_bump_coeffs(n_lon, n_lat, rng.uniform(0, 2 * math.pi),
                              math.acos(rng.uniform(-0.9, 0.9)), 5.0e5, 500.0)
    u = random_spectrum(rng, n_lon, n_lat, 3.0, VECTOR)
    v = random_spectrum(rng, n_lon, n_lat, 3.0, VECTOR)
    u *= 20.0 / coeff_norm(u)
    v *= 20.0 / coeff_norm(v)
    lon, colat = divergent_departure(rng, *grid0_points(n_lon, n_lat), 80.0, 1800.0)
    sample = np.sort(rng.choice(lon.size, n_sample, replace=False))
    tol = 1e-6 if dtype == "f32" else 1e-12
    return Workload("c3_%dx%d_%s" % (n_lon, n_lat, dtype), n_lon, n_lat,
                    np.stack([h, u, v]), lon, colat, tol, dtype, sample=sample)


ENSEMBLE_GRIDS = ((128, 64), (256, 128), (512, 256), (1024, 512))
SERVE_GRIDS = ((128, 64), (256, 128), (512, 256), (1024, 512), (2048, 1024))


def workload_member(seed: int, n_lon: int, n_lat: int, dtype: str = "f32",
                    dt: float = 3600.0, n_sample: int = 256) -> Workload:
    """One ensemble member or served request: fields (h, u, v) with |k|^-3 spectra,
    a seeded solid-body rotation angle alpha in [0, pi/2]."""
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(0.0, math.pi / 2)
    fields = [random_spectrum(rng, n_lon, n_lat, 3.0, p) for p in (SCALAR, VECTOR, VECTOR)]
    lon, colat = solid_body_departure(*grid0_points(n_lon, n_lat), alpha, U0_12DAY, dt)
    sample = np.sort(rng.choice(lon.size, min(n_sample, lon.size), replace=False))
    tol = 1e-6 if dtype == "f32" else 1e-12
    return Workload("member%d_%dx%d_%s" % (seed, n_lon, n_lat, dtype), n_lon, n_lat,
                    np.stack(fields), lon, colat, tol, dtype, sample=sample)


def workload_c4(n_per_size: int = 16) -> list[Workload]:
    """64 members, 16 at each of 128x64, 256x128, 512x256, 1024x512, FP32."""
    out = []
    for gi, (n_lon, n_lat) in enumerate(ENSEMBLE_GRIDS):
        for k in range(n_per_size):
            out.append(workload_member(4 + gi * n_per_size + k, n_lon, n_lat, "f32"))
    return out


def random_pr_spectrum(rng: np.random.Generator, M: int, N: int, decay: float) -> np.ndarray:
    """Partial-regularity DFS coefficients (index [m, n], n fastest, complex:
    cosine part + i sine part) with Gaussian entries of amplitude
    (1 + |k|)^-decay; zero outside each m's index range (n = 0..N for m = 0,
    0..N-1 for m = 1, 1..N-1 for even m, 1..N-2 for odd m) and no sine part at m = 0."""
    m = np.arange(M + 1)[:, None]
    n = np.arange(N + 1)[None, :]
    amp = (1.0 + np.sqrt(m * m + n * n)) ** (-decay)
    c = (rng.standard_normal((M + 1, N + 1)) + 1j * rng.standard_normal((M + 1, N + 1))) * amp
    lo = np.where(m == 0, 0, np.where(m == 1, 0, 1))
    hi = np.where(m == 0, N, np.where(m == 1, N - 1, np.where(m % 2 == 0, N - 1, N - 2)))
    c[(n < lo) | (n > hi)] = 0.0
    c[0, :] = c[0, :].real
    return c


def small_workload(seed: int, n_lon: int, n_lat: int, n_fields: int = 1, decay: float = 2.0,
                   dtype: str = "f64", tol: float | None = None,
                   points: str = "rotation") -> Workload:
    """Small seeded problems for parity tests (rotation or divergent points)."""
    rng = np.random.default_rng(seed)
    pars = [SCALAR, VECTOR, VECTOR, SCALAR]
    fields = [random_spectrum(rng, n_lon, n_lat, decay, pars[i % 4]) for i in range(n_fields)]
    ll, cc = grid0_points(n_lon, n_lat)
    if points == "rotation":
        lon, colat = solid_body_departure(ll, cc, rng.uniform(0, math.pi / 2), U0_12DAY, 3600.0)
    elif points == "divergent":
        lon, colat = divergent_departure(rng, ll, cc, 80.0, 1800.0)
    elif points == "uniform":
        lon = rng.uniform(0, 2 * math.pi, ll.size)
        colat = np.arccos(rng.uniform(-1, 1, ll.size))
    else:
        raise ValueError(points)
    if tol is None:
        tol = 1e-12 if dtype == "f64" else 1e-6
    return Workload("small%d_%dx%d" % (seed, n_lon, n_lat), n_lon, n_lat, np.stack(fields),
                    lon, colat, tol, dtype, sample=np.arange(lon.size))
