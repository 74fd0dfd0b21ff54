"""Parity of the CUDA path (through the C ABI) with the FP64 direct-sum oracle.

Acceptance (relative l-infinity over the checked points, per field, against
the oracle's real part): <= 1e-11 for FP64 plans at tol 1e-12 and <= 2e-5
for FP32 plans at tol 1e-6.  Other tolerances are checked at 10 x tol.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_01313_gb300 import build, synth

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11
TOL_F32 = 2e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def accept(dtype, tol):
    if dtype == "f64":
        return TOL_F64 if tol == 1e-12 else 10 * tol
    return TOL_F32 if tol >= 1e-6 else 20 * tol


def run_gpu(torch, wl, dtype=None, tol=None, lon=None, colat=None):
    from paper_2605_01313_gb300 import Plan
    dtype = dtype or wl.dtype
    tol = tol or wl.tol
    lon = wl.lon if lon is None else lon
    colat = wl.colat if colat is None else colat
    cd = torch.complex128 if dtype == "f64" else torch.complex64
    with Plan(wl.n_lon, wl.n_lat, tol, dtype, wl.n_fields) as plan:
        plan.set_points(torch.from_numpy(np.ascontiguousarray(lon)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(colat)).cuda())
        out = plan.execute(torch.from_numpy(wl.coeffs).to(cd).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def check_against_oracle(vals, wl, bound, sample=None, lon=None, colat=None):
    sample = wl.sample if sample is None else sample
    lon = wl.lon if lon is None else lon
    colat = wl.colat if colat is None else colat
    ref = oracle.evaluate(wl.coeffs, lon[sample], colat[sample])
    errs = []
    for f in range(wl.n_fields):
        e = oracle.rel_linf(vals[f][sample], ref[f].real)
        errs.append(e)
    assert max(errs) <= bound, (wl.name, errs, bound)
    return errs


# ------------------------------------------------------------------ the workloads

def test_c1_f64_all_points(torch_cuda):
    wl = synth.workload_c1()
    vals = run_gpu(torch_cuda, wl)
    check_against_oracle(vals, wl, TOL_F64)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_c2_three_fields(torch_cuda, dtype):
    wl = synth.workload_c2(dtype)
    vals = run_gpu(torch_cuda, wl)
    check_against_oracle(vals, wl, accept(dtype, wl.tol))


def test_c3_f32_full_size(torch_cuda):
    wl = synth.workload_c3("f32")
    vals = run_gpu(torch_cuda, wl)
    assert np.all(np.isfinite(vals))
    check_against_oracle(vals, wl, TOL_F32)


def test_c3_f64_full_size(torch_cuda):
    wl = synth.workload_c3("f64", n_sample=300)
    vals = run_gpu(torch_cuda, wl)
    check_against_oracle(vals, wl, TOL_F64)


@pytest.mark.parametrize("shift", [(110, 110, 110), (-110, -110, -110), (110, -110, 0)])
def test_c3_f64_scaled_coefficients(torch_cuda, shift):
    """FP64 plans compute in double-single arithmetic (pairs of FP32 numbers),
    yet keep their accuracy at any magnitude of the coefficients: the C3 fields
    times 2^k, far outside FP32's exponent range (each field with its own k in
    the mixed case), give exactly the unscaled values times 2^k, within 1e-11
    of the oracle."""
    wl = synth.workload_c3("f64", n_sample=200)
    base = run_gpu(torch_cuda, wl)
    s = np.array([math.ldexp(1.0, k) for k in shift])
    scaled = synth.Workload(wl.name, wl.n_lon, wl.n_lat, wl.coeffs * s[:, None, None], wl.lon,
                            wl.colat, wl.tol, "f64", sample=wl.sample)
    vals = run_gpu(torch_cuda, scaled)
    assert np.array_equal(vals, base * s[:, None])
    check_against_oracle(vals, scaled, TOL_F64)


# ------------------------------------------------------- sizes, fields, tolerances

@pytest.mark.parametrize("n_lon,n_lat", [(8, 4), (16, 8), (24, 12), (64, 32), (96, 48),
                                         (160, 80), (256, 128)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_small_grids_every_point(torch_cuda, n_lon, n_lat, dtype):
    for nf, pts in ((1, "rotation"), (3, "divergent"), (2, "uniform")):
        wl = synth.small_workload(100 + n_lon + nf, n_lon, n_lat, n_fields=nf, dtype=dtype,
                                  points=pts)
        vals = run_gpu(torch_cuda, wl)
        check_against_oracle(vals, wl, accept(dtype, wl.tol))


def test_f32_many_fields_whole_torus(torch_cuda):
    """Seven FP32 fields (more than one field group per bin) at points spread
    over the whole doubled torus, colatitude in [-pi, pi), so that bins on
    both seams (their tiles wrap around) are exercised with the rest."""
    rng = np.random.default_rng(41)
    base = synth.small_workload(41, 512, 256, n_fields=7, dtype="f32", decay=3.0)
    P = 40000
    lon = rng.uniform(0, 2 * math.pi, P)
    colat = rng.uniform(-math.pi, math.pi, P)
    # points piled up against the seams of both angles
    lon[:2000] = rng.uniform(-1e-3, 1e-3, 2000)
    colat[2000:4000] = rng.uniform(-1e-3, 1e-3, 2000)
    colat[4000:5000] = math.pi + rng.uniform(-1e-3, 1e-3, 1000)
    vals = run_gpu(torch_cuda, base, lon=lon, colat=colat)
    sample = np.concatenate([np.arange(0, 5000, 5), rng.choice(P, 1000, replace=False)])
    check_against_oracle(vals, base, TOL_F32, sample=sample, lon=lon, colat=colat)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("real", [False, True])
def test_largest_fine_grid(torch_cuda, dtype, real):
    """The largest grid a plan takes: 4096 x 4096 modes, fine grid 8192 x 8192
    (the wide forms of both FFT passes), one field, points everywhere."""
    from paper_2605_01313_gb300.nufft import Options
    rng = np.random.default_rng(71)
    n_lon, n_lat = 4096, 2048
    c = synth.random_spectrum(rng, n_lon, n_lat, 3.0, synth.SCALAR)[None]
    P = 20000
    lon = rng.uniform(0, 2 * math.pi, P)
    colat = rng.uniform(-math.pi, math.pi, P)
    tol = 1e-12 if dtype == "f64" else 1e-6
    from paper_2605_01313_gb300 import Plan
    import torch
    cd = torch.complex128 if dtype == "f64" else torch.complex64
    with Plan(n_lon, n_lat, tol, dtype, 1, options=Options.make(real_fields=real)) as plan:
        assert plan.params["n1"] == 8192 and plan.params["n2"] == 8192
        plan.set_points(torch.from_numpy(lon).cuda(), torch.from_numpy(colat).cuda())
        vals = plan.execute(torch.from_numpy(c).to(cd).cuda()).cpu().numpy()
    s = np.arange(0, P, 200)
    ref = oracle.evaluate(c, lon[s], colat[s])
    err = oracle.rel_linf(vals[0][s], ref[0].real)
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


def test_tolerance_sweep_monotone(torch_cuda):
    wl = synth.small_workload(7, 64, 32, n_fields=1, dtype="f64", points="uniform")
    ref = oracle.evaluate(wl.coeffs, wl.lon, wl.colat)[0].real
    prev = 1.0
    for tol in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14):
        err = oracle.rel_linf(run_gpu(torch_cuda, wl, tol=tol)[0], ref)
        assert err <= 10 * tol, (tol, err)
        assert err < prev or err < 1e-14, (tol, err, prev)
        prev = err
    for tol in (1e-2, 1e-4, 1e-6, 1e-7):
        err = oracle.rel_linf(run_gpu(torch_cuda, wl, dtype="f32", tol=tol)[0], ref)
        assert err <= max(10 * tol, 5e-6), (tol, err)


@pytest.mark.parametrize("n_points", [1, 2, 7, 31, 1000, 4097])
def test_ragged_point_counts(torch_cuda, n_points):
    rng = np.random.default_rng(n_points)
    wl = synth.small_workload(9, 64, 32, n_fields=2, dtype="f64")
    lon = rng.uniform(0, 2 * math.pi, n_points)
    colat = np.arccos(rng.uniform(-1, 1, n_points))
    vals = run_gpu(torch_cuda, wl, lon=lon, colat=colat)
    assert vals.shape == (2, n_points)
    check_against_oracle(vals, wl, TOL_F64, sample=np.arange(n_points), lon=lon, colat=colat)


# ------------------------------------------------------------------ edge cases

def test_edge_coordinates(torch_cuda):
    """Poles, seams, coordinates outside [0, 2pi) x [0, pi], fine-grid nodes and
    bin edges all match the oracle (which evaluates the same periodic series)."""
    wl = synth.small_workload(11, 64, 32, n_fields=1, dtype="f64")
    n1 = 128
    lon = np.array([0.0, 2 * math.pi, -math.pi, 7 * math.pi, 1e-17, -1e-17, 2 * math.pi * (1 - 1e-16),
                    math.pi, 2 * math.pi * 31 / n1, 2 * math.pi * 32 / n1, 2 * math.pi * 95.5 / n1,
                    3.0, 3.0, 3.0, 3.0, 1.0, 100.0, -100.0])
    colat = np.array([0.0, math.pi, 0.0, math.pi, 1.0, 2.0, 0.5, -0.3, math.pi + 0.3, 2 * math.pi,
                      -2 * math.pi, 1e-300, math.pi - 1e-16, 2 * math.pi * 16 / n1,
                      2 * math.pi * 15.5 / n1, 4.5, 50.0, -50.0])
    for dtype in ("f64", "f32"):
        vals = run_gpu(torch_cuda, wl, dtype=dtype, tol=1e-12 if dtype == "f64" else 1e-6,
                       lon=lon, colat=colat)
        check_against_oracle(vals, wl, TOL_F64 if dtype == "f64" else TOL_F32,
                             sample=np.arange(lon.size), lon=lon, colat=colat)


def test_non_finite_point_gives_nan_only_there(torch_cuda):
    wl = synth.small_workload(12, 32, 16, n_fields=2, dtype="f64")
    lon = wl.lon.copy()
    colat = wl.colat.copy()
    lon[5] = np.nan
    colat[9] = np.inf
    vals = run_gpu(torch_cuda, wl, lon=lon, colat=colat)
    bad = np.zeros(lon.size, bool)
    bad[[5, 9]] = True
    assert np.all(np.isnan(vals[:, bad]))
    good = np.nonzero(~bad)[0]
    check_against_oracle(vals, wl, TOL_F64, sample=good, lon=lon, colat=colat)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_single_modes_including_nyquist(torch_cuda, dtype):
    """One unit coefficient at (n0, m0) evaluates to cos(m0 phi + n0 theta).

    A lone mode at the corner of the band is the kernel's worst case (the 1-D
    band-edge error in both dimensions); the width rule keeps it within the
    same bound as every other input: 1e-11 at tol 1e-12."""
    n_lon, n_lat = 32, 16
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    rng = np.random.default_rng(13)
    lon = rng.uniform(-1, 7, 300)
    colat = rng.uniform(-1, 4, 300)
    bound = TOL_F64 if dtype == "f64" else TOL_F32
    for n0, m0 in [(0, 0), (3, -5), (n2 // 2 - 1, n1 // 2 - 1), (-(n2 // 2), -(n1 // 2)),
                   (-(n2 // 2), 4), (7, -(n1 // 2)), (n2 // 2 - 1, -(n1 // 2) + 1),
                   (-(n2 // 2) + 1, n1 // 2 - 1)]:
        c = np.zeros((1, n2, n1), np.complex128)
        c[0, n0 + n2 // 2, m0 + n1 // 2] = 1.0
        wl = synth.Workload("mode", n_lon, n_lat, c, lon, colat, 1e-12 if dtype == "f64" else 1e-6,
                            dtype)
        vals = run_gpu(torch_cuda, wl)
        want = np.cos(m0 * lon + n0 * colat)
        assert np.max(np.abs(vals[0] - want)) <= bound, (n0, m0)


def test_grid_point_reproduction(torch_cuda):
    """Coefficients interpolating samples on the doubled Grid [0] torus reproduce the
    samples at those points (exact reproduction up to the NUFFT tolerance)."""
    n_lon, n_lat = 64, 32
    n2, n1 = synth.coeff_shape(n_lon, n_lat)
    rng = np.random.default_rng(14)
    samples = rng.standard_normal((n2, n1))
    c = synth.torus_samples_to_coeffs(samples)
    th = (np.arange(n2) + 0.5) * (2 * math.pi / n2)
    ph = np.arange(n1) * (2 * math.pi / n1)
    tt, pp = np.meshgrid(th, ph, indexing="ij")
    wl = synth.Workload("repro", n_lon, n_lat, c[None], pp.ravel(), tt.ravel(), 1e-12, "f64")
    vals = run_gpu(torch_cuda, wl)
    assert np.max(np.abs(vals[0] - samples.ravel())) <= 1e-11 * np.max(np.abs(samples)) * 10


@pytest.mark.parametrize("parity", [synth.SCALAR, synth.VECTOR])
def test_dfs_symmetry(torch_cuda, parity):
    rng = np.random.default_rng(15)
    c = synth.random_spectrum(rng, 128, 64, 2.0, parity)[None]
    lon = rng.uniform(0, 2 * math.pi, 2000)
    colat = np.arccos(rng.uniform(-1, 1, 2000))
    wl = synth.Workload("sym", 128, 64, c, lon, colat, 1e-12, "f64")
    a = run_gpu(torch_cuda, wl)[0]
    b = run_gpu(torch_cuda, wl, lon=lon + math.pi, colat=-colat)[0]
    assert np.max(np.abs(b - parity * a)) <= 2e-11 * np.max(np.abs(a))


def test_zonal_flow_analytic(torch_cuda):
    """The steady zonal geostrophic flow's exact coefficients give the analytic h, u, v
    at the departure points."""
    alpha = math.pi / 2 - 0.05
    n_lon, n_lat = 64, 32
    c = np.stack(synth.zonal_flow_coeffs(n_lon, n_lat, alpha))
    lon, colat = synth.solid_body_departure(*synth.grid0_points(n_lon, n_lat), alpha,
                                            synth.U0_12DAY, 5000.0)
    wl = synth.Workload("tc2", n_lon, n_lat, c, lon, colat, 1e-12, "f64")
    vals = run_gpu(torch_cuda, wl)
    for f, want in enumerate(synth.zonal_flow_values(lon, colat, alpha)):
        assert np.max(np.abs(vals[f] - want)) <= 1e-11 * np.max(np.abs(want))


# ------------------------------------------------------------------ API behaviour

@pytest.mark.parametrize("n_fields", [1, 3, 5])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_host_variants_match_device(torch_cuda, n_fields, dtype):
    """The host-buffer calls (one field: one transform; several fields:
    pipelined field by field) give the device path's values bit for bit."""
    from paper_2605_01313_gb300 import Plan
    wl = synth.small_workload(16, 128, 64, n_fields=n_fields, dtype=dtype)
    dev = run_gpu(torch_cuda, wl)
    cd = np.complex128 if dtype == "f64" else np.complex64
    with Plan(wl.n_lon, wl.n_lat, wl.tol, dtype, n_fields) as plan:
        for _ in range(2):
            plan.set_points_host(wl.lon, wl.colat)
            host = plan.execute_host(wl.coeffs.astype(cd))
            assert np.array_equal(dev, host)


@pytest.mark.parametrize("real", [True, False])
@pytest.mark.parametrize("n_fields", [1, 3])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_execute_points_host_matches_the_two_calls(torch_cuda, n_fields, dtype, real):
    """execute_points_host (points and coefficients from the host in one call;
    for FP32 plans of several fields field 0's transform runs over every fine
    row before the points are sorted) gives the values of set_points_host
    followed by execute_host bit for bit, leaves the points set for a later
    execute, and agrees with the oracle; the points change between calls."""
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.nufft import Options
    torch = torch_cuda
    cd = np.complex128 if dtype == "f64" else np.complex64
    tol = 1e-12 if dtype == "f64" else 1e-6
    bound = 1e-11 if dtype == "f64" else 2e-5
    wls = [synth.small_workload(seed, 128, 64, n_fields=n_fields, dtype=dtype) for seed in (5, 6)]
    with Plan(128, 64, tol, dtype, n_fields, options=Options.make(real_fields=real)) as plan:
        for wl in wls:
            c = wl.coeffs.astype(cd)
            joint = plan.execute_points_host(wl.lon, wl.colat, c)
            plan.set_points_host(wl.lon, wl.colat)
            apart = plan.execute_host(c)
            assert np.array_equal(joint, apart)
            plan.execute_points_host(wl.lon, wl.colat, c)
            dev = plan.execute(torch.from_numpy(c).cuda()).cpu().numpy()
            assert np.array_equal(dev, joint)
            s_ = wl.sample[:64]
            ref = oracle.evaluate(wl.coeffs, wl.lon[s_], wl.colat[s_])
            for f in range(n_fields):
                assert oracle.rel_linf(joint[f][s_], ref[f].real) <= bound


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_host_execute_real_plan_stages_what_it_reads(torch_cuda, dtype):
    """A real-field plan's execute_host copies only the columns m >= 0 and the
    Nyquist row and column: two different coefficient arrays in a row (white
    noise in every entry, so that a part missed by the copy would come from the
    first array) give the device path's values for each."""
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.nufft import Options, dfsnufft_plan_host_copy_bytes
    torch = torch_cuda
    n_lon, n_lat, F = 64, 32, 3
    rng = np.random.default_rng(41)
    lon = rng.uniform(0, 2 * math.pi, 3000)
    colat = np.arccos(rng.uniform(-1, 1, 3000))
    cd = np.complex128 if dtype == "f64" else np.complex64
    arrays = [(rng.standard_normal((F, 2 * n_lat, n_lon)) +
               1j * rng.standard_normal((F, 2 * n_lat, n_lon))).astype(cd) for _ in range(2)]
    tol = 1e-12 if dtype == "f64" else 1e-6
    with Plan(n_lon, n_lat, tol, dtype, F, options=Options.make(real_fields=True)) as plan:
        plan.set_points(torch.from_numpy(lon).cuda(), torch.from_numpy(colat).cuda())
        dev = [plan.execute(torch.from_numpy(c).cuda()).cpu().numpy() for c in arrays]
        plan.set_points_host(lon, colat)
        host = [plan.execute_host(c) for c in arrays]
        nb = dfsnufft_plan_host_copy_bytes(plan._h)
        # the staging buffer is shared with interpolate_grid, queued without a
        # wait: the next host copy must not overtake its reads
        rd = torch.float64 if dtype == "f64" else torch.float32
        samples = torch.from_numpy(rng.standard_normal((F, n_lat, n_lon))).to(rd).cuda()
        from_grid = plan.interpolate_grid(samples, [1, -1, -1])
        again = plan.execute_host(arrays[0])
        from_grid_dev = plan.interpolate_grid(samples, [1, -1, -1]).cpu().numpy()
        assert np.array_equal(from_grid.cpu().numpy(), from_grid_dev)
    for d, h in zip(dev, host):
        assert np.array_equal(d, h)
    assert np.array_equal(again, dev[0])
    cs = 16 if dtype == "f64" else 8
    rows, half = F * 2 * n_lat, cs * n_lon // 2
    assert nb["coeffs_h2d"] == (rows - 1) * (half + cs) + half + F * (half + cs)
    assert nb["points_h2d"] == 16 * 3000 and nb["values_d2h"] == cs // 2 * F * 3000


def test_repeatable_and_resettable(torch_cuda):
    from paper_2605_01313_gb300 import Plan
    torch = torch_cuda
    wl = synth.small_workload(17, 64, 32, n_fields=2, dtype="f64")
    rng = np.random.default_rng(5)
    coeffs = torch.from_numpy(wl.coeffs).cuda()
    with Plan(wl.n_lon, wl.n_lat, 1e-12, "f64", 2) as plan:
        lo, co = torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda()
        plan.set_points(lo, co)
        a = plan.execute(coeffs).cpu().numpy()
        b = plan.execute(coeffs).cpu().numpy()
        assert np.array_equal(a, b)
        big_lon = rng.uniform(0, 2 * math.pi, 20000)
        big_col = np.arccos(rng.uniform(-1, 1, 20000))
        plan.set_points(torch.from_numpy(big_lon).cuda(), torch.from_numpy(big_col).cuda())
        c = plan.execute(coeffs).cpu().numpy()
        check_against_oracle(c, wl, TOL_F64, sample=np.arange(0, 20000, 97), lon=big_lon,
                             colat=big_col)
        plan.set_points(lo, co)
        d = plan.execute(coeffs).cpu().numpy()
        assert np.array_equal(a, d)


def test_errors(torch_cuda):
    from paper_2605_01313_gb300 import Plan, nufft
    torch = torch_cuda
    plan = Plan(64, 32, 1e-12, "f64", 1)
    coeffs = torch.zeros((1, 64, 64), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(nufft.DfsError) as ei:
        nufft.dfsnufft_execute(plan._h, coeffs.data_ptr(), out.data_ptr())
    assert ei.value.status == nufft.ERR_NO_POINTS
    with pytest.raises(nufft.DfsError) as ei:
        nufft.dfsnufft_set_points(plan._h, 0, 0, 0)
    assert ei.value.status == nufft.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        plan.execute(coeffs.to(torch.complex64))
    plan.destroy()
    with pytest.raises(nufft.DfsError) as ei:
        nufft.dfsnufft_plan_create(63, 32, 1e-12, "f64", 1, 0)
    assert ei.value.status == nufft.ERR_INVALID_ARG


def test_two_plans_two_streams(torch_cuda):
    from paper_2605_01313_gb300 import Plan
    torch = torch_cuda
    wl = synth.small_workload(18, 128, 64, n_fields=3, dtype="f32")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    lo, co = torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda()
    cf = torch.from_numpy(wl.coeffs).to(torch.complex64).cuda()
    torch.cuda.synchronize()
    p1 = Plan(wl.n_lon, wl.n_lat, wl.tol, "f32", 3, stream=s1)
    p2 = Plan(wl.n_lon, wl.n_lat, wl.tol, "f32", 3, stream=s2)
    p1.set_points(lo, co)
    p2.set_points(lo, co)
    with torch.cuda.stream(s1):
        o1 = torch.empty((3, lo.numel()), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s2):
        o2 = torch.empty((3, lo.numel()), dtype=torch.float32, device="cuda")
    p1.execute(cf, o1)
    p2.execute(cf, o2)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    p1.destroy()
    p2.destroy()
