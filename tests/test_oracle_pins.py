"""Pins of the oracle against what the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself: a closed form, a
library special case, an independent evaluation route, an invariant of the
doubled sphere, or a physical balance.  The last group plants mistakes in
copies of the oracle and checks that the pins catch them.
"""
import math

import numpy as np
import pytest

from paper_2605_01313_gb300 import synth


def _rand_points(rng, n, full_torus=False):
    lon = rng.uniform(0.0, 2.0 * math.pi, n)
    if full_torus:
        colat = rng.uniform(-math.pi, 2.0 * math.pi, n)
    else:
        colat = np.arccos(rng.uniform(-1.0, 1.0, n))
    return lon, colat


# ---------------------------------------------------------------- P5: single modes

@pytest.mark.parametrize("n_lon,n_lat", [(8, 4), (64, 32), (256, 128)])
def test_single_mode_closed_form(oracle_mod, n_lon, n_lat):
    """A coefficient array with one unit entry at (n0, m0) gives exp(i(m0 phi + n0 theta))."""
    rng = np.random.default_rng(10)
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    lon, colat = _rand_points(rng, 64, full_torus=True)
    modes = [(0, 0), (1, 0), (0, 1), (-1, 3), (n2 // 2 - 1, n1 // 2 - 1),
             (-(n2 // 2) + 1, -(n1 // 2) + 1), (-(n2 // 2), -(n1 // 2)), (2, -(n1 // 2))]
    for n0, m0 in modes:
        c = np.zeros((n2, n1), dtype=np.complex128)
        c[n0 + n2 // 2, m0 + n1 // 2] = 1.0
        got = oracle_mod.evaluate(c, lon, colat)
        want = np.cos(m0 * lon + n0 * colat) + 1j * np.sin(m0 * lon + n0 * colat)
        assert np.max(np.abs(got - want)) < 1e-12, (n0, m0)


# ------------------------------------------------------------- P6: tiny brute force

@pytest.mark.parametrize("n_lon,n_lat", [(8, 4), (16, 8)])
def test_brute_force_matrix(oracle_mod, n_lon, n_lat):
    """Direct C sum == dense NUDFT matrix product on tiny grids (arbitrary complex
    coefficients, no symmetry, points anywhere on the doubled torus)."""
    rng = np.random.default_rng(11)
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    c = rng.standard_normal((n2, n1)) + 1j * rng.standard_normal((n2, n1))
    lon, colat = _rand_points(rng, 200, full_torus=True)
    got = oracle_mod.evaluate(c, lon, colat)
    want = oracle_mod.nudft_matrix(c, lon, colat)
    assert np.max(np.abs(got - want)) < 1e-13 * np.sum(np.abs(c))


@pytest.mark.parametrize("n_lon,n_lat", [(8, 4), (16, 8), (32, 16)])
def test_cossin_route(oracle_mod, n_lon, n_lat):
    """Eq. 5.4 then Eq. 5.3 equals the real cos/sin form Eq. 4.6-4.7 evaluated
    directly, and the complex form is real."""
    rng = np.random.default_rng(12)
    N, M = n_lat - 1, n_lon // 2 - 1
    fc = rng.standard_normal((N + 1, M + 1))
    fs = rng.standard_normal((N + 1, M + 1))
    c = oracle_mod.complex_from_cossin(fc, fs, n_lon, n_lat)
    lon, colat = _rand_points(rng, 300)
    got = oracle_mod.evaluate(c, lon, colat)
    want = oracle_mod.eval_cossin(fc, fs, lon, colat)
    scale = np.sum(np.abs(fc)) + np.sum(np.abs(fs))
    assert np.max(np.abs(got.real - want)) < 1e-13 * scale
    assert np.max(np.abs(got.imag)) < 1e-13 * scale


def test_cossin_route_has_scalar_parity(oracle_mod):
    """The standard DFS basis (even m <-> cos n theta, odd m <-> sin n theta) gives
    c_{-n,m} = (-1)^m c_{n,m}: the scalar symmetry of Sec. 4."""
    rng = np.random.default_rng(13)
    n_lon, n_lat = 16, 8
    fc = rng.standard_normal((n_lat, n_lon // 2))
    fs = rng.standard_normal((n_lat, n_lon // 2))
    c = oracle_mod.complex_from_cossin(fc, fs, n_lon, n_lat)
    sym = synth.symmetrize(c, synth.SCALAR)
    assert np.max(np.abs(sym - c)) < 1e-15


# ------------------------------------------------------- P1: grid-point reproduction

@pytest.mark.parametrize("n_lon,n_lat", [(8, 4), (16, 8)])
def test_grid_point_reproduction(oracle_mod, n_lon, n_lat):
    """Coefficients obtained by inverting the sampling on the doubled Grid [0] torus
    (explicit DFT sums, half-cell offset in theta) reproduce the samples."""
    rng = np.random.default_rng(14)
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    samples = rng.standard_normal((n2, n1))
    th = (np.arange(n2) + 0.5) * (2 * math.pi / n2)
    ph = np.arange(n1) * (2 * math.pi / n1)
    n = np.arange(n2) - n2 // 2
    m = np.arange(n1) - n1 // 2
    et = np.exp(-1j * np.outer(n, th))          # (N2 modes, N2 samples)
    ep = np.exp(-1j * np.outer(ph, m))          # (N1 samples, N1 modes)
    c = et @ samples @ ep / (n1 * n2)
    tt, pp = np.meshgrid(th, ph, indexing="ij")
    got = oracle_mod.evaluate(c, pp.ravel(), tt.ravel()).reshape(n2, n1)
    assert np.max(np.abs(got - samples)) < 1e-13
    # the generator's FFT route to the same coefficients agrees
    c_gen = synth.torus_samples_to_coeffs(samples)
    assert np.max(np.abs(c_gen - c)) < 1e-14


def test_grid_point_reproduction_arrival_grid(oracle_mod):
    """Samples of a real scalar field on the sphere's Grid [0] (through Cartesian
    coordinates) are reproduced at every arrival point."""
    rng = np.random.default_rng(15)
    n_lon, n_lat = 32, 16
    a = rng.standard_normal(4)

    def field(lon, colat):
        x, y, z = np.sin(colat) * np.cos(lon), np.sin(colat) * np.sin(lon), np.cos(colat)
        return np.exp(a[0] * x + a[1] * y) * np.cos(2 * z + a[2]) + a[3] * x * y * z

    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    th = (np.arange(n2) + 0.5) * (2 * math.pi / n2)
    ph = np.arange(n1) * (2 * math.pi / n1)
    tt, pp = np.meshgrid(th, ph, indexing="ij")
    c = synth.torus_samples_to_coeffs(field(pp, tt))
    lon, colat = synth.grid0_points(n_lon, n_lat)
    got = oracle_mod.evaluate(c, lon, colat)
    assert np.max(np.abs(got - field(lon, colat))) < 1e-12


# ------------------------------------------------- P2: steady zonal geostrophic flow

def test_zonal_flow_coefficients_exact(oracle_mod):
    """The closed-form coefficients of the tilted zonal flow evaluate to the pointwise
    formulas for h, u, v."""
    rng = np.random.default_rng(16)
    lon, colat = _rand_points(rng, 500)
    for alpha in (0.0, math.pi / 4, math.pi / 2 - 0.05):
        coeffs = synth.zonal_flow_coeffs(16, 8, alpha)
        vals = synth.zonal_flow_values(lon, colat, alpha)
        for c, want in zip(coeffs, vals):
            got = oracle_mod.evaluate(c, lon, colat)
            scale = max(np.max(np.abs(want)), 1.0)
            assert np.max(np.abs(got.real - want)) < 1e-13 * scale
            assert np.max(np.abs(got.imag)) < 1e-13 * scale


def _tangent_basis(lon, colat):
    e_lon = np.stack([-np.sin(lon), np.cos(lon), np.zeros_like(lon)], -1)
    # northward unit vector = -d r / d colat
    e_north = -np.stack([np.cos(colat) * np.cos(lon), np.cos(colat) * np.sin(lon),
                         -np.sin(colat)], -1)
    return e_lon, e_north


def test_zonal_flow_is_steady():
    """Steadiness of the generator's flow under Eq. 2.1a with the Coriolis vector along
    the tilted axis: P[(V.grad)V + 2 Omega k x V] + g grad h = 0, finite differences."""
    rng = np.random.default_rng(17)
    alpha = math.pi / 2 - 0.05
    lon, colat = _rand_points(rng, 50)
    colat = np.clip(colat, 0.2, math.pi - 0.2)
    a = synth.EARTH_RADIUS

    def wind3d(xyz):
        lo, co = synth.from_xyz(xyz)
        _, u, v = synth.zonal_flow_values(lo, co, alpha)
        el, en = _tangent_basis(lo, co)
        return u[:, None] * el + v[:, None] * en

    def height(xyz):
        lo, co = synth.from_xyz(xyz)
        return synth.zonal_flow_values(lo, co, alpha)[0]

    r = synth.to_xyz(lon, colat)
    V = wind3d(r)
    eps = 1e-6
    sp = np.linalg.norm(V, axis=1)
    vh = V / sp[:, None]
    dV = (wind3d(r + eps * vh) - wind3d(r - eps * vh)) / (2 * eps) * (sp / a)[:, None]
    gh = np.zeros_like(r)
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        gh[:, k] = (height(r + e) - height(r - e)) / (2 * eps) / a
    k_axis = synth.rotation_axis(alpha)
    cor = 2 * synth.EARTH_OMEGA * np.cross(k_axis[None, :], V)
    total = dV + cor + synth.GRAVITY * gh
    total -= np.sum(total * r, axis=1, keepdims=True) * r      # tangential part
    scale = np.max(np.abs(cor))
    assert np.max(np.abs(total)) < 1e-6 * scale


# -------------------------------------------------- P3: solid-body rotation, degree 1

def test_solid_body_rotation_degree_one(oracle_mod):
    """f = n.r has coefficients only at |n|, |m| <= 1 (written out by hand); at the
    departure points of a solid-body rotation it equals n.(R(-w dt) r_A), with the
    rotation built independently by scipy."""
    from scipy.spatial.transform import Rotation
    n_lon, n_lat = 64, 32
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    nv = np.array([0.3, -0.7, 0.5])
    c = np.zeros((n2, n1), dtype=np.complex128)
    r0, q0 = n2 // 2, n1 // 2
    # x = sin(t)cos(p), y = sin(t)sin(p), z = cos(t), expanded in exp(i(n t + m p))
    for sn in (1, -1):
        for sm in (1, -1):
            c[r0 + sn, q0 + sm] += nv[0] * (-0.25j * sn)             # x
            c[r0 + sn, q0 + sm] += nv[1] * (-0.25 * sn * sm)         # y
        c[r0 + sn, q0] += nv[2] * 0.5                                 # z
    alpha, dt = math.pi / 4, 3600.0
    lon_a, colat_a = synth.grid0_points(n_lon, n_lat)
    lon_d, colat_d = synth.solid_body_departure(lon_a, colat_a, alpha, synth.U0_12DAY, dt)
    got = oracle_mod.evaluate(c, lon_d, colat_d)
    angle = synth.U0_12DAY * dt / synth.EARTH_RADIUS
    axis = np.array([-math.sin(alpha), 0.0, math.cos(alpha)])
    rot = Rotation.from_rotvec(-angle * axis)
    want = rot.apply(synth.to_xyz(lon_a, colat_a)) @ nv
    assert np.max(np.abs(got.real - want)) < 1e-13
    assert np.max(np.abs(got.imag)) < 1e-13


# ----------------------------------------------------------- P4: DFS symmetry

@pytest.mark.parametrize("parity", [synth.SCALAR, synth.VECTOR])
def test_dfs_symmetry(oracle_mod, parity):
    """f(phi + pi, -theta) = +f(phi, theta) for scalars and -f for wind components
    (Sec. 4), and the fields are real."""
    rng = np.random.default_rng(18)
    c = synth.random_spectrum(rng, 32, 16, 2.0, parity)
    lon, colat = _rand_points(rng, 200)
    a = oracle_mod.evaluate(c, lon, colat)
    b = oracle_mod.evaluate(c, lon + math.pi, -colat)
    scale = np.max(np.abs(a))
    assert np.max(np.abs(b - parity * a)) < 1e-13 * scale
    assert np.max(np.abs(a.imag)) < 1e-13 * scale


def test_batched_fields_match_single(oracle_mod):
    rng = np.random.default_rng(19)
    c = np.stack([synth.random_spectrum(rng, 16, 8, 2.0, p) for p in (1, -1, -1)])
    lon, colat = _rand_points(rng, 50)
    got = oracle_mod.evaluate(c, lon, colat)
    for i in range(3):
        assert np.array_equal(got[i], oracle_mod.evaluate(c[i], lon, colat))


def test_rel_linf():
    assert oracle_rel(np.array([1.0, 2.0]), np.array([1.0, 4.0])) == 0.5


def oracle_rel(a, b):
    import oracle
    return oracle.rel_linf(a, b)


# ---------------------------------------------- planted mistakes are caught by pins

def _single_mode_ok(evaluate, n_lon=16, n_lat=8):
    rng = np.random.default_rng(20)
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    lon, colat = _rand_points(rng, 40, full_torus=True)
    for n0, m0 in [(1, 0), (0, 1), (-3, 2), (2, -5)]:
        c = np.zeros((n2, n1), dtype=np.complex128)
        c[n0 + n2 // 2, m0 + n1 // 2] = 1.0
        want = np.exp(1j * (m0 * lon + n0 * colat))
        if np.max(np.abs(evaluate(c, lon, colat) - want)) > 1e-12:
            return False
    return True


def _brute_ok(evaluate, n_lon=8, n_lat=4):
    import oracle
    rng = np.random.default_rng(21)
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    c = rng.standard_normal((n2, n1)) + 1j * rng.standard_normal((n2, n1))
    lon, colat = _rand_points(rng, 30, full_torus=True)
    return np.max(np.abs(evaluate(c, lon, colat) - oracle.nudft_matrix(c, lon, colat))) < 1e-12


def test_pins_accept_the_oracle(oracle_mod):
    assert _single_mode_ok(oracle_mod.evaluate)
    assert _brute_ok(oracle_mod.evaluate)


@pytest.mark.parametrize("mistake", ["transposed", "conjugate_sign", "swapped_axes",
                                     "off_by_one_centre", "dropped_row", "dropped_imag"])
def test_pins_catch_planted_mistakes(oracle_mod, mistake):
    ev = oracle_mod.evaluate

    def bad(c, lon, colat):
        if mistake == "transposed":
            return ev(np.ascontiguousarray(c.T) if c.shape[0] == c.shape[1]
                      else np.ascontiguousarray(c.T.reshape(c.shape)), lon, colat)
        if mistake == "conjugate_sign":
            return np.conj(ev(np.conj(c), lon, colat))
        if mistake == "swapped_axes":
            return ev(c, colat, lon)
        if mistake == "off_by_one_centre":
            return ev(np.roll(c, 1, axis=1), lon, colat)
        if mistake == "dropped_row":
            c2 = np.array(c)
            c2[-1] = 0.0
            return ev(c2, lon, colat)
        if mistake == "dropped_imag":
            return ev(c.real.astype(np.complex128), lon, colat)
        raise AssertionError(mistake)

    assert not (_single_mode_ok(bad) and _brute_ok(bad))


# ------------------------------------------- partial-regularity DFS coefficients (Sec. 4)

def _pr_coeffs(rng, N, M):
    pc = rng.standard_normal((N + 1, M + 1))
    ps = rng.standard_normal((N + 1, M + 1))
    ps[:, 0] = 0.0
    return pc, ps


@pytest.mark.parametrize("N,M", [(12, 9), (8, 5), (31, 20)])
def test_pr_map_matches_direct_pr_evaluation(oracle_mod, N, M):
    """The standard coefficients from pr_to_std evaluate (Eq. 4.6-4.7) to the same
    field as the partial-regularity basis functions of Sec. 4 evaluated
    directly (trigonometric products, no product-to-sum step)."""
    rng = np.random.default_rng(500 + N)
    pc, ps = _pr_coeffs(rng, N, M)
    lon, colat = _rand_points(rng, 400, full_torus=True)
    fc, fs = oracle_mod.pr_to_std(pc, ps)
    direct = oracle_mod.eval_pr(pc, ps, lon, colat)
    assert np.max(np.abs(oracle_mod.eval_cossin(fc, fs, lon, colat) - direct)) < 1e-12


def test_pr_expansion_is_pole_regular(oracle_mod):
    """Every m >= 1 term carries a sin(theta) factor, so a field without m = 0
    vanishes at both poles, whichever longitude (Sec. 4, property 3)."""
    rng = np.random.default_rng(503)
    pc, ps = _pr_coeffs(rng, 14, 10)
    pc[:, 0] = 0.0
    fc, fs = oracle_mod.pr_to_std(pc, ps)
    lon = rng.uniform(0, 2 * math.pi, 50)
    for pole in (0.0, math.pi):
        th = np.full(50, pole)
        assert np.max(np.abs(oracle_mod.eval_pr(pc, ps, lon, th))) < 1e-12
        assert np.max(np.abs(oracle_mod.eval_cossin(fc, fs, lon, th))) < 1e-12


def test_pr_printed_f0_for_even_m_would_fail(oracle_mod):
    """The list in Sec. 4 prints f~_{0,m} = 0 for even m >= 2; the pin above
    rejects that value (the sin(theta) sin(theta) term has a constant part)."""
    rng = np.random.default_rng(504)
    pc, ps = _pr_coeffs(rng, 12, 6)
    fc, fs = oracle_mod.pr_to_std(pc, ps)
    fc_printed, fs_printed = fc.copy(), fs.copy()
    for m in range(2, 7, 2):
        fc_printed[0, m] = fs_printed[0, m] = 0.0
    lon, colat = _rand_points(rng, 200)
    direct = oracle_mod.eval_pr(pc, ps, lon, colat)
    assert np.max(np.abs(oracle_mod.eval_cossin(fc_printed, fs_printed, lon, colat)
                         - direct)) > 1e-3


def test_pr_through_complex_map_and_direct_sum(oracle_mod):
    """The whole chain the GPU takes: partial-regularity -> standard (Sec. 4) ->
    complex (Eq. 5.4) -> direct sum (Eq. 5.3) equals the direct PR evaluation."""
    rng = np.random.default_rng(505)
    n_lon, n_lat = 32, 16
    N, M = 14, 15
    pc, ps = _pr_coeffs(rng, N, M)
    fc, fs = oracle_mod.pr_to_std(pc, ps)
    c = oracle_mod.complex_from_cossin(fc, fs, n_lon, n_lat)
    lon, colat = _rand_points(rng, 300, full_torus=True)
    v = oracle_mod.evaluate(c[None], lon, colat)[0]
    assert np.max(np.abs(v.imag)) < 1e-12
    assert np.max(np.abs(v.real - oracle_mod.eval_pr(pc, ps, lon, colat))) < 1e-12


# ------------------------------------------------ grid values -> coefficients (Sec. 3-4)

@pytest.mark.parametrize("n_lon,n_lat", [(16, 8), (32, 16), (64, 32)])
def test_grid_to_coeffs_recovers_band_limited_fields(oracle_mod, n_lon, n_lat):
    """Real DFS-symmetric fields (scalar and vector parity, Nyquist zero) sampled
    on the arrival grid by the direct sum give back their own coefficients."""
    rng = np.random.default_rng(600 + n_lon)
    c = np.stack([synth.random_spectrum(rng, n_lon, n_lat, 1.5, par)
                  for par in (synth.SCALAR, synth.VECTOR, synth.VECTOR)])
    lon, colat = synth.grid0_points(n_lon, n_lat)
    vals = oracle_mod.evaluate(c, lon, colat).real.reshape(3, n_lat, n_lon)
    got = oracle_mod.grid_to_coeffs(vals, [1, -1, -1])
    assert np.max(np.abs(got - c)) < 1e-13


def test_grid_to_coeffs_reproduces_samples_and_parity(oracle_mod):
    """Arbitrary samples: the coefficients' series passes through every sample of
    the arrival grid, and on the other half of the doubled torus equals the
    parity extension f(phi + pi, -theta) = +-f(phi, theta)."""
    rng = np.random.default_rng(610)
    n_lon, n_lat = 24, 12
    s = rng.standard_normal((2, n_lat, n_lon))
    c = oracle_mod.grid_to_coeffs(s, [1, -1])
    lon, colat = synth.grid0_points(n_lon, n_lat)
    got = oracle_mod.evaluate(c, lon, colat).real.reshape(2, n_lat, n_lon)
    assert np.max(np.abs(got - s)) < 1e-12
    lon2 = lon + math.pi
    back = oracle_mod.evaluate(c, lon2, -colat).real.reshape(2, n_lat, n_lon)
    assert np.max(np.abs(back[0] - s[0])) < 1e-12
    assert np.max(np.abs(back[1] + s[1])) < 1e-12


@pytest.mark.parametrize("mistake", ["no_half_cell", "wrong_parity", "no_shift"])
def test_grid_to_coeffs_pins_catch_mistakes(oracle_mod, mistake):
    """Copies of grid_to_coeffs with one plausible mistake fail the recovery pin."""
    rng = np.random.default_rng(620)
    n_lon, n_lat = 16, 8
    c = np.stack([synth.random_spectrum(rng, n_lon, n_lat, 1.5, synth.VECTOR)])
    lon, colat = synth.grid0_points(n_lon, n_lat)
    vals = oracle_mod.evaluate(c, lon, colat).real.reshape(1, n_lat, n_lon)
    n2, n1 = 2 * n_lat, n_lon
    th = (np.arange(n2) + (0.0 if mistake == "no_half_cell" else 0.5)) * (math.pi / n_lat)
    ph = np.arange(n1) * (2 * math.pi / n1)
    n = np.arange(n2) - n2 // 2
    m = np.arange(n1) - n1 // 2
    ext = np.empty((n2, n1))
    ext[:n_lat] = vals[0]
    for j in range(n_lat, n2):
        row = vals[0][n2 - 1 - j]
        if mistake != "no_shift":
            row = np.roll(row, -(n1 // 2))
        ext[j] = (1.0 if mistake == "wrong_parity" else -1.0) * row
    bad = np.exp(-1j * np.outer(n, th)) @ ext @ np.exp(-1j * np.outer(ph, m)) / (n1 * n2)
    assert np.max(np.abs(bad - c[0])) > 1e-3


def test_grid_to_coeffs_conjugate_symmetry_and_antiperiodic_nyquist_row(oracle_mod):
    """Real samples give c_{-n,-m} = conj c_{n,m}; on the half-cell theta grid the
    sum is antiperiodic in n (e^{-i N2 theta_j} = -1), so the Nyquist row of the
    columns -m is minus the conjugate of the row at m (the GPU transform writes
    the columns m < 0 from these two facts)."""
    rng = np.random.default_rng(630)
    n_lon, n_lat = 16, 6
    s = rng.standard_normal((1, n_lat, n_lon))
    c = oracle_mod.grid_to_coeffs(s, [-1])[0]
    N2, N1 = 2 * n_lat, n_lon
    for m in range(1, N1 // 2):
        qm, qn = N1 // 2 + m, N1 // 2 - m
        for n in range(-N2 // 2 + 1, N2 // 2):
            assert abs(c[N2 // 2 - n, qn] - np.conj(c[N2 // 2 + n, qm])) < 1e-14
        assert abs(c[0, qn] + np.conj(c[0, qm])) < 1e-14
    # the row formula at n = +N2/2 (outside the array) is minus the row at -N2/2
    th = (np.arange(N2) + 0.5) * (math.pi / n_lat)
    ph = np.arange(N1) * (2 * math.pi / N1)
    ext = np.empty((N2, N1))
    ext[:n_lat] = s[0]
    for j in range(n_lat, N2):
        ext[j] = -np.roll(s[0][N2 - 1 - j], -(N1 // 2))
    top = np.exp(-1j * (N2 // 2) * th) @ ext @ np.exp(-1j * np.outer(ph, np.arange(N1) - N1 // 2))
    assert np.max(np.abs(top / (N1 * N2) + c[0])) < 1e-14
