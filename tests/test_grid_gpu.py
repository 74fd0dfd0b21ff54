"""Grid values to coefficients on the GPU (dfsnufft_grid_to_coeffs) and the
whole interpolation step from the arrival grid (dfsnufft_interpolate_grid),
against the oracle's plain doubled-torus Fourier sums."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_01313_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def plan_for(n_lon, n_lat, dtype, F, real=True, members=1):
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.nufft import Options
    tol = 1e-12 if dtype == "f64" else 1e-6
    return Plan(n_lon, n_lat, tol, dtype, F, n_members=members,
                options=Options.make(real_fields=real))


# (32, 1024) and (32, 2048): columns of 2048 and 4096 doubled rows, the longest
# the theta pass takes (blocks of 2 and 1 columns in FP64, 4 and 2 in FP32)
@pytest.mark.parametrize("n_lon,n_lat", [(16, 8), (64, 32), (128, 64), (512, 256), (256, 512),
                                         (32, 1024), (32, 2048)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_grid_to_coeffs_matches_oracle(torch_cuda, n_lon, n_lat, dtype):
    torch = torch_cuda
    rng = np.random.default_rng(800 + n_lon + n_lat)
    s = rng.standard_normal((3, n_lat, n_lon))
    par = [1, -1, -1]
    rd = torch.float64 if dtype == "f64" else torch.float32
    with plan_for(n_lon, n_lat, dtype, 3) as plan:
        c = plan.grid_to_coeffs(torch.from_numpy(s).to(rd).cuda(), par).cpu().numpy()
    ref = oracle.grid_to_coeffs(s.astype(np.float32).astype(np.float64)
                                if dtype == "f32" else s, par)
    # white-noise samples: both sides carry rounding of order eps log2(N1 N2) times
    # the samples' size, against coefficients of size 1/sqrt(N1 N2)
    err = np.max(np.abs(c - ref)) / np.max(np.abs(ref))
    assert err <= (1e-12 if dtype == "f64" else 2e-6), err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_interpolate_grid_reproduces_arrival_samples(torch_cuda, dtype):
    """With the departure points at the arrival points the step returns the samples."""
    torch = torch_cuda
    n_lon, n_lat = 128, 64
    rng = np.random.default_rng(810)
    s = rng.standard_normal((2, n_lat, n_lon))
    lon, colat = synth.grid0_points(n_lon, n_lat)
    rd = torch.float64 if dtype == "f64" else torch.float32
    with plan_for(n_lon, n_lat, dtype, 2) as plan:
        plan.set_points(torch.from_numpy(lon).cuda(), torch.from_numpy(colat).cuda())
        v = plan.interpolate_grid(torch.from_numpy(s).to(rd).cuda(), [1, -1]).cpu().numpy()
    err = np.max(np.abs(v.reshape(2, n_lat, n_lon) - s)) / np.max(np.abs(s))
    assert err <= (1e-11 if dtype == "f64" else 2e-5), err


@pytest.mark.parametrize("real", [True, False])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_interpolate_grid_band_limited_fields(torch_cuda, dtype, real):
    """Band-limited fields (scalar and wind parity) sampled on the arrival grid are
    carried to departure points exactly as their series evaluates there, by a
    real-field plan (which stages only the columns m >= 0) and a general one."""
    torch = torch_cuda
    wl = synth.workload_member(820, 256, 128, dtype, n_sample=400)
    c = wl.coeffs
    lon_a, colat_a = synth.grid0_points(256, 128)
    s = oracle.evaluate(c, lon_a, colat_a).real.reshape(3, 128, 256)
    rd = torch.float64 if dtype == "f64" else torch.float32
    with plan_for(256, 128, dtype, 3, real=real) as plan:
        plan.set_points(torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda())
        v = plan.interpolate_grid(torch.from_numpy(s).to(rd).cuda(), [1, -1, -1]).cpu().numpy()
    ref = oracle.evaluate(c, wl.lon[wl.sample], wl.colat[wl.sample])
    err = max(oracle.rel_linf(v[f][wl.sample], ref[f].real) for f in range(3))
    assert err <= (1e-11 if dtype == "f64" else 2e-5), err


def test_grid_batched_members_and_errors(torch_cuda):
    from paper_2605_01313_gb300 import nufft
    torch = torch_cuda
    rng = np.random.default_rng(830)
    s = rng.standard_normal((2, 2, 32, 64))
    with plan_for(64, 32, "f64", 2, members=2) as plan:
        c = plan.grid_to_coeffs(torch.from_numpy(s).cuda(), [1, -1]).cpu().numpy()
        for k in range(2):
            ref = oracle.grid_to_coeffs(s[k], [1, -1])
            assert np.max(np.abs(c[k] - ref)) <= 1e-13 * np.max(np.abs(ref))
        with pytest.raises(nufft.DfsError) as ei:
            plan.grid_to_coeffs(torch.from_numpy(s).cuda(), [1, 0])
        assert ei.value.status == nufft.ERR_INVALID_ARG
    with plan_for(24, 12, "f64", 1) as plan:             # not powers of two
        with pytest.raises(nufft.DfsError) as ei:
            plan.grid_to_coeffs(torch.zeros((1, 12, 24), dtype=torch.float64, device="cuda"),
                                [1])
        assert ei.value.status == nufft.ERR_UNSUPPORTED


def test_grid_to_coeffs_f64_scaled_samples(torch_cuda):
    """FP64 plans transform in double-single arithmetic: samples times 2^-110
    and 2^+110 (one field each, far outside FP32's exponent range) give exactly
    the unscaled coefficients times the same powers of two, within the FP64
    bound of the oracle."""
    torch = torch_cuda
    n_lon, n_lat = 512, 256
    rng = np.random.default_rng(840)
    s = rng.standard_normal((n_lat, n_lon))
    k = np.array([math.ldexp(1.0, -110), math.ldexp(1.0, 110)])
    with plan_for(n_lon, n_lat, "f64", 2) as plan:
        base = plan.grid_to_coeffs(torch.from_numpy(np.stack([s, s])).cuda(), [1, -1]).cpu().numpy()
        c = plan.grid_to_coeffs(torch.from_numpy(np.stack([s * k[0], s * k[1]])).cuda(),
                                [1, -1]).cpu().numpy()
    for f in range(2):
        assert np.array_equal(c[f], base[f] * k[f])
        ref = oracle.grid_to_coeffs(s[None], [(1, -1)[f]])[0]
        assert np.max(np.abs(base[f] - ref)) <= 1e-12 * np.max(np.abs(ref))
