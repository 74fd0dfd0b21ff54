"""Departure points (Eq. 2.4) and the vector rotation Q (Sec. 2) on the GPU,
against the FP64 oracle (oracle/departure.py), through the C ABI.

Tolerances.  FP64 runs the same arithmetic as the oracle in another order:
1e-12 rad.  FP32 iterates in single precision relative to the arrival point:
the quintic sums carry about 2.6 u |W| (sum of |weights| per direction about
1.6, unit roundoff u = 6e-8) and the great-circle step a few u of the
displacement, so the position error is a few 1e-7 of the largest displacement;
the test allows 5e-6 of it."""
import math

import numpy as np
import pytest

from oracle import departure as dep
from paper_2605_01313_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def xyz(lon, colat):
    s = np.sin(colat)
    return np.stack([s * np.cos(lon), s * np.sin(lon), np.cos(colat)], axis=-1)


def rigid_field(axis, omega, n_lon, n_lat):
    """East/north components of omega axis x r on Grid [0]."""
    lon, colat = dep.arrival_points(n_lon, n_lat)
    r = xyz(lon, colat)
    v = omega * np.cross(axis, r)
    east = np.stack([-np.sin(lon), np.cos(lon), np.zeros_like(lon)], axis=-1)
    north = np.stack([-np.cos(colat) * np.cos(lon), -np.cos(colat) * np.sin(lon),
                      np.sin(colat)], axis=-1)
    return np.stack([np.sum(v * east, 1).reshape(n_lat, n_lon),
                     np.sum(v * north, 1).reshape(n_lat, n_lon)])


def inputs(n_lon, n_lat, seed, omega=60.0):
    rng = np.random.default_rng(seed)
    t, p = rng.uniform(0.2, 1.3), rng.uniform(0, 2 * math.pi)
    axis = np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])
    w = rigid_field(axis, omega, n_lon, n_lat)
    # a smooth arrival term of a few m/s (Omega x r-like plus a tilt)
    wa = 0.05 * rigid_field(np.array([0.0, 0.0, 1.0]), omega, n_lon, n_lat)
    wa[1] += 2.0 * rng.standard_normal() * np.cos(np.arange(n_lon) * 2 * math.pi / n_lon)[None, :]
    return w, wa


def chord(lon1, colat1, lon2, colat2):
    return np.linalg.norm(xyz(lon1, colat1) - xyz(lon2, colat2), axis=-1)


def run(torch, w, wa, dt_over_a, iterations, dtype):
    from paper_2605_01313_gb300 import nufft
    rd = torch.float64 if dtype == "f64" else torch.float32
    wt = torch.from_numpy(w).to(rd).cuda().contiguous()
    wat = None if wa is None else torch.from_numpy(wa).to(rd).cuda().contiguous()
    lon, colat = nufft.departure_points(wt, dt_over_a, iterations, wat)
    torch.cuda.synchronize()
    return lon.cpu().numpy(), colat.cpu().numpy()


def rounded(a, dtype):
    return a.astype(np.float32).astype(np.float64) if dtype == "f32" else a


@pytest.mark.parametrize("n_lon,n_lat", [(128, 64), (96, 48), (6, 3), (40, 21)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_departure_points_match_oracle(torch_cuda, n_lon, n_lat, dtype):
    """Every arrival point, displacements up to about three cells (across the
    poles for the rows next to them), four iterations."""
    w, wa = inputs(n_lon, n_lat, 900 + n_lon)
    # at most three cells and 0.2 rad: the iteration stays a contraction
    dt_over_a = min(3.0 * math.pi / n_lat, 0.2) / 60.0
    w, wa = rounded(w, dtype), rounded(wa, dtype)
    lon, colat = run(torch_cuda, w, wa, dt_over_a, 4, dtype)
    ol, oc = dep.departure_points(w, wa, dt_over_a, 4)
    la, ca = dep.arrival_points(n_lon, n_lat)
    disp = np.max(chord(ol, oc, la, ca))
    err = np.max(chord(lon, colat, ol, oc))
    assert np.all((lon >= 0) & (lon < 2 * math.pi))
    # where the displacement reaches past the first row's colatitude, some of
    # its departure points lie across the pole (longitude turned by about half a turn)
    turn = np.abs(np.angle(np.exp(1j * (ol[:n_lon] - la[:n_lon]))))
    if disp > math.pi / n_lat:
        assert np.any(turn > 0.5 * math.pi)
    bound = 1e-12 if dtype == "f64" else 5e-6 * disp
    assert err <= bound, (err, disp)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_departure_points_full_grid_sampled(torch_cuda, dtype):
    """2048 x 1024, the bench's configuration (three iterations, 1800 s over the
    Earth's radius, TC2-like speeds), checked at seeded samples and the pole rows."""
    n_lon, n_lat = 2048, 1024
    w, wa = inputs(n_lon, n_lat, 950, omega=40.0)
    w, wa = rounded(w, dtype), rounded(wa, dtype)
    dt_over_a = 1800.0 / synth.EARTH_RADIUS
    lon, colat = run(torch_cuda, w, wa, dt_over_a, 3, dtype)
    rng = np.random.default_rng(951)
    index = np.concatenate([rng.integers(0, n_lon * n_lat, 3000), np.arange(0, n_lon, 7),
                            n_lon * n_lat - 1 - np.arange(0, n_lon, 5)])
    ol, oc = dep.departure_points(w, wa, dt_over_a, 3, index=index)
    la, ca = dep.arrival_points(n_lon, n_lat)
    disp = np.max(chord(ol, oc, la[index], ca[index]))
    err = np.max(chord(lon[index], colat[index], ol, oc))
    assert err <= (1e-12 if dtype == "f64" else 5e-6 * disp), (err, disp)


def test_departure_one_iteration_and_members(torch_cuda):
    """One iteration is the great-circle step from the grid values; two members
    with different fields and no arrival term."""
    torch = torch_cuda
    from paper_2605_01313_gb300 import nufft
    n_lon, n_lat = 64, 32
    w0, _ = inputs(n_lon, n_lat, 960)
    w1, _ = inputs(n_lon, n_lat, 961)
    dt_over_a = 0.02 / 60.0
    wt = torch.from_numpy(np.stack([w0, w1])).cuda()
    for iters in (1, 5):
        lon, colat = nufft.departure_points(wt, dt_over_a, iters)
        lon, colat = lon.cpu().numpy(), colat.cpu().numpy()
        assert lon.shape == (2, n_lon * n_lat)
        for k, w in enumerate((w0, w1)):
            ol, oc = dep.departure_points(w, None, dt_over_a, iters)
            assert np.max(chord(lon[k], colat[k], ol, oc)) <= 1e-12


def test_departure_zero_wind_stays_at_arrival(torch_cuda):
    torch = torch_cuda
    from paper_2605_01313_gb300 import nufft
    w = torch.zeros((2, 16, 32), dtype=torch.float64, device="cuda")
    lon, colat = nufft.departure_points(w, 1.0, 3)
    la, ca = dep.arrival_points(32, 16)
    assert np.array_equal(lon.cpu().numpy(), la)
    assert np.array_equal(colat.cpu().numpy(), ca)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rotate_to_arrival_matches_oracle_in_place_with_stride(torch_cuda, dtype):
    torch = torch_cuda
    from paper_2605_01313_gb300 import nufft
    n_lon, n_lat, F, members = 64, 32, 3, 2
    P = n_lon * n_lat
    rng = np.random.default_rng(970)
    deps = [dep.departure_points(*inputs(n_lon, n_lat, 971 + m), 0.1 / 60.0, 3)
            for m in range(members)]
    lon_d = np.stack([d[0] for d in deps])
    colat_d = np.stack([d[1] for d in deps])
    vals = rounded(rng.standard_normal((members, F, P)), dtype)
    rd = torch.float64 if dtype == "f64" else torch.float32
    vt = torch.from_numpy(vals).to(rd).cuda()
    flat = vt.view(-1)
    u, v = flat[P:], flat[2 * P:]
    nufft.rotate_to_arrival(n_lon, n_lat, torch.from_numpy(lon_d).cuda(),
                            torch.from_numpy(colat_d).cuda(), u, v, stride=F * P,
                            members=members, u_a=u, v_a=v)
    got = vt.cpu().numpy()
    la, ca = dep.arrival_points(n_lon, n_lat)
    # |p|, |q| <= 1: a few roundings of p, q and the 2 x 2 product times |u| + |v| (< 10)
    bound = 4e-14 if dtype == "f64" else 1e-5
    for m in range(members):
        eu, ev = dep.rotate_to_arrival(vals[m, 1], vals[m, 2], la, ca, lon_d[m], colat_d[m])
        assert np.max(np.abs(got[m, 1] - eu)) <= bound
        assert np.max(np.abs(got[m, 2] - ev)) <= bound
        assert np.array_equal(got[m, 0], vals[m, 0])          # untouched field


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_semi_lagrangian_step_chain(torch_cuda, dtype):
    """Departure points, then values of (h, u, v) at them from arrival-grid
    samples, then (u, v) rotated to the arrival frame: the whole step against
    the oracle's chain (departure points, grid-to-coefficient sums, direct
    evaluation, Q)."""
    import oracle
    torch = torch_cuda
    from paper_2605_01313_gb300 import Plan, nufft
    from paper_2605_01313_gb300.nufft import Options
    n_lon, n_lat = 128, 64
    alpha = 0.7
    la, ca = dep.arrival_points(n_lon, n_lat)
    h, u, v = synth.zonal_flow_values(la, ca, alpha)
    samples = np.stack([h, u, v]).reshape(3, n_lat, n_lon)
    w, wa = synth.zonal_flow_settls_terms(la, ca, alpha, 3600.0)
    w = rounded(w.reshape(2, n_lat, n_lon), dtype)
    wa = rounded(wa.reshape(2, n_lat, n_lon), dtype)
    dt_over_a = 3600.0 / synth.EARTH_RADIUS
    rd = torch.float64 if dtype == "f64" else torch.float32
    pq = torch.empty((2, n_lon * n_lat), dtype=rd, device="cuda")
    lon_d, colat_d = nufft.departure_points(torch.from_numpy(w).to(rd).cuda(), dt_over_a, 3,
                                            torch.from_numpy(wa).to(rd).cuda(), pq_out=pq)
    tol = 1e-12 if dtype == "f64" else 1e-6
    with Plan(n_lon, n_lat, tol, dtype, 3, options=Options.make(real_fields=True)) as plan:
        plan.set_points(lon_d, colat_d)
        vals = plan.interpolate_grid(torch.from_numpy(samples).to(rd).cuda(), [1, -1, -1])
        nufft.rotate_to_arrival(n_lon, n_lat, None, None, vals[1], vals[2],
                                u_a=vals[1], v_a=vals[2], pq=pq)
        got = vals.cpu().numpy()
    s = np.concatenate([np.arange(0, n_lon * n_lat, 13), np.arange(n_lon)])
    ol, oc = dep.departure_points(w, wa, dt_over_a, 3, index=s)
    sq = samples.astype(np.float32).astype(np.float64) if dtype == "f32" else samples
    ref = oracle.evaluate(oracle.grid_to_coeffs(sq, [1, -1, -1]), ol, oc).real
    ru, rv = dep.rotate_to_arrival(ref[1], ref[2], la[s], ca[s], ol, oc)
    ref = np.stack([ref[0], ru, rv])
    for f in range(3):
        err = np.max(np.abs(got[f][s] - ref[f])) / np.max(np.abs(ref[f]))
        assert err <= (1e-11 if dtype == "f64" else 2e-5), (f, err)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rotation_from_departure_pq(torch_cuda, dtype):
    """p and q written by the departure kernel for its final points: the
    rotation read from them equals the oracle's Q at those points, two members."""
    torch = torch_cuda
    from paper_2605_01313_gb300 import nufft
    n_lon, n_lat, members = 96, 48, 2
    P = n_lon * n_lat
    w = np.stack([rounded(inputs(n_lon, n_lat, 980 + m)[0], dtype) for m in range(members)])
    rd = torch.float64 if dtype == "f64" else torch.float32
    pq = torch.empty((members, 2, P), dtype=rd, device="cuda")
    lon, colat = nufft.departure_points(torch.from_numpy(w).to(rd).cuda(), 0.15 / 60.0, 3,
                                        pq_out=pq)
    rng = np.random.default_rng(981)
    vals = rounded(rng.standard_normal((members, 2, P)), dtype)
    vt = torch.from_numpy(vals).to(rd).cuda()
    flat = vt.view(-1)
    ua, va = nufft.rotate_to_arrival(n_lon, n_lat, None, None, flat, flat[P:], stride=2 * P,
                                     members=members, pq=pq)
    ua = ua.cpu().numpy()
    va = va.cpu().numpy()
    lon, colat = lon.cpu().numpy(), colat.cpu().numpy()
    la, ca = dep.arrival_points(n_lon, n_lat)
    p_, q_ = pq.cpu().numpy()[:, 0], pq.cpu().numpy()[:, 1]
    bound = 4e-14 if dtype == "f64" else 1e-5
    for m in range(members):
        p_ref, q_ref = dep.rotation_pq(la, ca, lon[m], colat[m])
        assert np.max(np.abs(p_[m] - p_ref)) <= bound / 4
        assert np.max(np.abs(q_[m] - q_ref)) <= bound / 4
        eu, ev = dep.rotate_to_arrival(vals[m, 0], vals[m, 1], la, ca, lon[m], colat[m])
        assert np.max(np.abs(ua[m * 2 * P:m * 2 * P + P] - eu)) <= bound
        assert np.max(np.abs(va[m * 2 * P:m * 2 * P + P] - ev)) <= bound
