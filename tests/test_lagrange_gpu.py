"""The Lagrange interpolation comparator (dfsnufft_lagrange_interp) on the GPU
against its FP64 oracle (oracle/lagrange.py), through the C ABI.

Tolerances.  The kernel reduces positions exactly (fractions of a turn in
fixed point); the oracle forms x = phi n / (2 pi) in FP64, off by up to
2^-52 |x| cells (|x| < 700 here: 1.6e-13 cells), which moves a value by at most
sum |L'| sum |L| (< 6 x 1.6) times that times the largest sample; with the
sums' own rounding, FP64 allows 2e-12 of the largest sample.  FP32: the sums in
single precision plus the offset rounded to FP32 (6e-8 of a cell): 2e-6 of the
largest sample for the random samples used here."""
import math

import numpy as np
import pytest

from oracle import lagrange as lag
from paper_2605_01313_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def run(torch, samples, parity, lon, colat, order, dtype):
    from paper_2605_01313_gb300 import nufft
    rd = torch.float64 if dtype == "f64" else torch.float32
    out = nufft.lagrange_interp(torch.from_numpy(samples).to(rd).cuda(), parity,
                                torch.from_numpy(lon).cuda(), torch.from_numpy(colat).cuda(),
                                order)
    return out.cpu().numpy()


@pytest.mark.parametrize("n_lon,n_lat", [(64, 32), (6, 3), (48, 20), (256, 128)])
@pytest.mark.parametrize("order", [3, 5])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_lagrange_matches_oracle(torch_cuda, n_lon, n_lat, order, dtype):
    if n_lon <= order:
        pytest.skip("grid narrower than the stencil")
    rng = np.random.default_rng(700 + n_lon + order)
    F = 3
    s = rng.standard_normal((F, n_lat, n_lon))
    if dtype == "f32":
        s = s.astype(np.float32).astype(np.float64)
    P = 5000
    # any real coordinate: the doubled torus and whole turns, points near both poles
    lon = rng.uniform(-7.0, 13.0, P)
    colat = np.concatenate([rng.uniform(-4.0, 7.0, P - 400), rng.uniform(0, 0.05, 200),
                            math.pi - rng.uniform(0, 0.05, 200)])
    par = [1, -1, -1]
    got = run(torch_cuda, s, par, lon, colat, order, dtype)
    bound = (2e-12 if dtype == "f64" else 2e-6) * np.max(np.abs(s))
    for f in range(F):
        ref = lag.interp_lagrange(s[f], par[f], lon, colat, order)
        assert np.max(np.abs(got[f] - ref)) <= bound, (f, np.max(np.abs(got[f] - ref)))


def test_lagrange_reproduces_nodes_and_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2605_01313_gb300 import nufft
    from oracle import departure as dep
    n_lon, n_lat = 32, 16
    rng = np.random.default_rng(710)
    s = rng.standard_normal((1, n_lat, n_lon))
    la, ca = dep.arrival_points(n_lon, n_lat)
    got = run(torch, s, [1], la, ca, 5, "f64")
    # a node's index position phi n / (2 pi) is an integer only up to FP64
    # rounding, so the weights are the unit vector up to a few 1e-15
    assert np.max(np.abs(got[0] - s[0].ravel())) < 1e-13
    t = torch.from_numpy(s).cuda()
    pts = torch.from_numpy(la).cuda()
    for order, par in ((4, [1]), (5, [0])):
        with pytest.raises(nufft.DfsError) as ei:
            nufft.lagrange_interp(t, par, pts, pts, order)
        assert ei.value.status == nufft.ERR_INVALID_ARG
    # non-finite and out-of-range coordinates give NaN, the rest is unaffected
    bad = torch.tensor([float("nan"), float("inf"), 2.0 ** 60, 0.5], dtype=torch.float64,
                       device="cuda")
    v = nufft.lagrange_interp(t, [1], bad, torch.full_like(bad, 0.7), 3).cpu().numpy()
    assert np.all(np.isnan(v[0, :3])) and np.isfinite(v[0, 3])
