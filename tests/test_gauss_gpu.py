"""Samples on a Gauss-Legendre latitude grid (DFSNUFFT_GAUSS_GRID) on the GPU,
against the FP64 oracle (oracle/gauss.py) through the C ABI.

Tolerances.  The latitude solve's matrices have condition numbers below 5 at
these sizes (cos and sin bases at the Gauss nodes), so the coefficients carry a
few units of rounding of the GEMM's precision: FP64 1e-12 and FP32 (the
tensor-core solve with TF32 operands split into two parts, FP32-level) 1e-5 of
the largest coefficient; values at departure points are then bounded as the
interpolation tests bound them (1e-11 FP64, 2e-5 FP32, relative l-inf)."""
import math

import numpy as np
import pytest

import oracle
from oracle import gauss
from paper_2605_01313_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def gl_plan(n_lon, n_lat, dtype, F, real=True, members=1):
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.nufft import Options
    tol = 1e-12 if dtype == "f64" else 1e-6
    return Plan(n_lon, n_lat, tol, dtype, F, n_members=members,
                options=Options.make(real_fields=real, gauss=True))


def grid_points(colat, n_lon):
    cc, ll = np.meshgrid(colat, np.arange(n_lon) * 2 * math.pi / n_lon, indexing="ij")
    return ll.ravel(), cc.ravel()


@pytest.mark.parametrize("n_lat", [8, 64, 512])
def test_nodes_are_the_gauss_legendre_nodes(torch_cuda, n_lat):
    with gl_plan(2 * n_lat, n_lat, "f64", 1) as plan:
        th = plan.latitudes()
    z, _ = np.polynomial.legendre.leggauss(n_lat)
    assert np.max(np.abs(np.cos(th) - np.sort(z)[::-1])) < 1e-14
    assert np.all(np.diff(th) > 0)


@pytest.mark.parametrize("n_lon,n_lat", [(16, 8), (64, 32), (256, 128), (512, 256)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_coefficients_match_oracle(torch_cuda, n_lon, n_lat, dtype):
    torch = torch_cuda
    rng = np.random.default_rng(850 + n_lon)
    s = rng.standard_normal((3, n_lat, n_lon))
    if dtype == "f32":
        s = s.astype(np.float32).astype(np.float64)
    par = [1, -1, -1]
    rd = torch.float64 if dtype == "f64" else torch.float32
    with gl_plan(n_lon, n_lat, dtype, 3, real=False) as plan:
        th = plan.latitudes()
        c = plan.grid_to_coeffs(torch.from_numpy(s).to(rd).cuda(), par).cpu().numpy()
    ref = gauss.gl_to_coeffs(s, par, th)
    err = np.max(np.abs(c - ref)) / np.max(np.abs(ref))
    assert err <= (1e-12 if dtype == "f64" else 1e-5), err


@pytest.mark.parametrize("real", [True, False])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_interpolation_from_gauss_samples(torch_cuda, dtype, real):
    """Band-limited fields sampled on the Gauss grid are carried to departure
    points as their series evaluates there (real-field and general plans)."""
    torch = torch_cuda
    wl = synth.workload_member(860, 256, 128, dtype, n_sample=400)
    with gl_plan(256, 128, dtype, 3, real=real) as plan:
        th = plan.latitudes()
        la, ca = grid_points(th, 256)
        s = oracle.evaluate(wl.coeffs, la, ca).real.reshape(3, 128, 256)
        rd = torch.float64 if dtype == "f64" else torch.float32
        plan.set_points(torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda())
        v = plan.interpolate_grid(torch.from_numpy(s).to(rd).cuda(), [1, -1, -1]).cpu().numpy()
    ref = oracle.evaluate(wl.coeffs, wl.lon[wl.sample], wl.colat[wl.sample])
    err = max(oracle.rel_linf(v[f][wl.sample], ref[f].real) for f in range(3))
    assert err <= (1e-11 if dtype == "f64" else 2e-5), err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_arbitrary_samples_real_and_general_plans_agree(torch_cuda, dtype):
    """White-noise samples (the interpolant's Nyquist terms non-zero): the real-
    field plan's staging keeps Re v of the full interpolant, as the general plan
    and the oracle's series do."""
    torch = torch_cuda
    rng = np.random.default_rng(870)
    n_lon, n_lat = 64, 32
    s = rng.standard_normal((2, n_lat, n_lon))
    if dtype == "f32":
        s = s.astype(np.float32).astype(np.float64)
    P = 3000
    lon = rng.uniform(0, 2 * math.pi, P)
    colat = rng.uniform(0, math.pi, P)
    rd = torch.float64 if dtype == "f64" else torch.float32
    vals = {}
    for real in (True, False):
        with gl_plan(n_lon, n_lat, dtype, 2, real=real) as plan:
            th = plan.latitudes()
            plan.set_points(torch.from_numpy(lon).cuda(), torch.from_numpy(colat).cuda())
            vals[real] = plan.interpolate_grid(torch.from_numpy(s).to(rd).cuda(),
                                               [1, -1]).cpu().numpy()
    ref = oracle.evaluate(gauss.gl_to_coeffs(s, [1, -1], th), lon, colat).real
    bound = 1e-11 if dtype == "f64" else 2e-5
    for real in (True, False):
        for f in range(2):
            err = np.max(np.abs(vals[real][f] - ref[f])) / np.max(np.abs(ref[f]))
            assert err <= bound, (real, f, err)


def test_members_and_unsupported_sizes(torch_cuda):
    torch = torch_cuda
    from paper_2605_01313_gb300 import Plan, nufft
    from paper_2605_01313_gb300.nufft import Options
    rng = np.random.default_rng(880)
    s = rng.standard_normal((2, 2, 16, 32))
    with gl_plan(32, 16, "f64", 2, real=False, members=2) as plan:
        th = plan.latitudes()
        c = plan.grid_to_coeffs(torch.from_numpy(s).cuda(), [1, -1]).cpu().numpy()
    for k in range(2):
        ref = gauss.gl_to_coeffs(s[k], [1, -1], th)
        assert np.max(np.abs(c[k] - ref)) <= 1e-12 * np.max(np.abs(ref))
    with pytest.raises(nufft.DfsError) as ei:
        Plan(24, 12, 1e-6, "f32", 1, options=Options.make(gauss=True))
    assert ei.value.status == nufft.ERR_UNSUPPORTED


@pytest.mark.parametrize("real", [True, False])
def test_unaligned_output_gives_the_same_coefficients(torch_cuda, real):
    """The coefficient mapping writes two modes of a row as one 16-byte store
    when the output is 16-byte aligned and one at a time otherwise: an output
    that starts one complex element into a buffer must get the same bits."""
    torch = torch_cuda
    n_lon, n_lat = 256, 128
    rng = np.random.default_rng(4242)
    s = torch.from_numpy(rng.standard_normal((3, n_lat, n_lon))).to(torch.float32).cuda()
    par = [1, -1, -1]
    with gl_plan(n_lon, n_lat, "f32", 3, real=real) as plan:
        aligned = plan.grid_to_coeffs(s, par).cpu()
        n = aligned.numel()
        buf = torch.zeros(n + 1, dtype=aligned.dtype, device="cuda")
        out = buf[1:].view(aligned.shape)
        assert out.data_ptr() % 16 == 8
        shifted = plan.grid_to_coeffs(s, par, out=out).cpu()
    assert torch.equal(torch.view_as_real(aligned), torch.view_as_real(shifted))

