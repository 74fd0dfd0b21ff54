"""Fields given by partial-regularity DFS coefficients (Sec. 4) on the GPU
(dfsnufft_execute_pr), against the oracle's map (pr_to_std, complex_from_cossin)
and direct sum, and against the direct evaluation of the expansion."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_01313_gb300 import build, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-12, 1e-11), "f32": (1e-6, 2e-5)}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def run_pr(torch, prs, lon, colat, n_lon, n_lat, dtype):
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.nufft import Options
    cd = torch.complex128 if dtype == "f64" else torch.complex64
    tol = TOL[dtype][0]
    with Plan(n_lon, n_lat, tol, dtype, prs.shape[0],
              options=Options.make(real_fields=True)) as plan:
        plan.set_points(torch.from_numpy(lon).cuda(), torch.from_numpy(colat).cuda())
        out = plan.execute_pr(torch.from_numpy(prs).to(cd).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def reference(pr, lon, colat, n_lon, n_lat):
    """Oracle route: partial-regularity -> standard -> complex -> direct sum."""
    pc = np.ascontiguousarray(pr.real.T)
    ps = np.ascontiguousarray(pr.imag.T)
    fc, fs = oracle.pr_to_std(pc, ps)
    c = oracle.complex_from_cossin(fc, fs, n_lon, n_lat)
    return oracle.evaluate(c[None], lon, colat)[0].real


@pytest.mark.parametrize("n_lon,n_lat,M,N", [(64, 32, 31, 30), (64, 32, 20, 9), (128, 64, 63, 62),
                                             (256, 128, 100, 126), (512, 256, 255, 254)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_pr_matches_oracle(torch_cuda, n_lon, n_lat, M, N, dtype):
    rng = np.random.default_rng(700 + n_lon + M)
    prs = np.stack([synth.random_pr_spectrum(rng, M, N, 2.0) for _ in range(2)])
    P = 2000
    lon = rng.uniform(-1.0, 2 * math.pi + 1.0, P)
    colat = rng.uniform(-math.pi, 2 * math.pi, P)
    vals = run_pr(torch_cuda, prs, lon, colat, n_lon, n_lat, dtype)
    s = np.arange(0, P, 4)
    for f in range(2):
        ref = reference(prs[f], lon[s], colat[s], n_lon, n_lat)
        assert oracle.rel_linf(vals[f][s], ref) <= TOL[dtype][1]


def test_pr_matches_direct_expansion_and_poles(torch_cuda):
    """Against the basis functions of Sec. 4 evaluated directly; at the poles a
    field without m = 0 vanishes (the expansion's regularity)."""
    rng = np.random.default_rng(710)
    M, N = 20, 28
    pr = synth.random_pr_spectrum(rng, M, N, 1.5)
    lon = rng.uniform(0, 2 * math.pi, 600)
    colat = np.concatenate([rng.uniform(0, math.pi, 500), np.zeros(50), np.full(50, math.pi)])
    vals = run_pr(torch_cuda, pr[None], lon, colat, 64, 32, "f64")[0]
    direct = oracle.eval_pr(pr.real.T.copy(), pr.imag.T.copy(), lon, colat)
    assert oracle.rel_linf(vals, direct) <= 1e-11
    pr0 = pr.copy()
    pr0[0, :] = 0.0
    vals0 = run_pr(torch_cuda, pr0[None], lon[500:], colat[500:], 64, 32, "f64")[0]
    assert np.max(np.abs(vals0)) <= 1e-11 * np.abs(pr).sum()


def test_pr_errors(torch_cuda):
    from paper_2605_01313_gb300 import Plan, nufft
    torch = torch_cuda
    rng = np.random.default_rng(711)
    lon = torch.from_numpy(rng.uniform(0, 6, 100)).cuda()
    colat = torch.from_numpy(rng.uniform(0, 3, 100)).cuda()
    pr = torch.zeros((1, 10, 12), dtype=torch.complex128, device="cuda")
    with Plan(64, 32, 1e-12, "f64", 1) as plan:         # general plan: not allowed
        plan.set_points(lon, colat)
        with pytest.raises(nufft.DfsError) as ei:
            plan.execute_pr(pr)
        assert ei.value.status == nufft.ERR_INVALID_ARG
    with Plan(64, 32, 1e-12, "f64", 1, options=nufft.Options.make(real_fields=True)) as plan:
        plan.set_points(lon, colat)
        big = torch.zeros((1, 33, 12), dtype=torch.complex128, device="cuda")   # M = 32 > 31
        with pytest.raises(nufft.DfsError) as ei:
            plan.execute_pr(big)
        assert ei.value.status == nufft.ERR_INVALID_ARG
        tall = torch.zeros((1, 10, 33), dtype=torch.complex128, device="cuda")  # N = 32 > 31
        with pytest.raises(nufft.DfsError) as ei:
            plan.execute_pr(tall)
        assert ei.value.status == nufft.ERR_INVALID_ARG
        plan.execute_pr(pr)
        plan.check()


def test_pr_f64_scaled_inputs(torch_cuda):
    """Partial-regularity input of an FP64 plan scaled by 2^-120 and 2^+120 (one
    field each): the values scale exactly, and stay within 1e-11 of the oracle."""
    rng = np.random.default_rng(712)
    M, N = 255, 254
    pr = synth.random_pr_spectrum(rng, M, N, 2.0)
    P = 1500
    lon = rng.uniform(0, 2 * math.pi, P)
    colat = rng.uniform(0, math.pi, P)
    base = run_pr(torch_cuda, pr[None], lon, colat, 512, 256, "f64")[0]
    s = np.array([math.ldexp(1.0, -120), math.ldexp(1.0, 120)])
    vals = run_pr(torch_cuda, pr[None] * s[:, None, None], lon, colat, 512, 256, "f64")
    idx = np.arange(0, P, 5)
    ref = reference(pr, lon[idx], colat[idx], 512, 256)
    for f in range(2):
        assert np.array_equal(vals[f], base * s[f])
        assert oracle.rel_linf(vals[f][idx], ref * s[f]) <= 1e-11
