"""Plan options on the GPU, against the FP64 oracle: real-field plans
(DFSNUFFT_REAL_FIELDS), unsorted points (DFSNUFFT_KEEP_ORDER), oversampling 4,
kernel width and bin size.

A real-field plan reads the columns m >= 0, the Nyquist column and the
Nyquist row only; its values are Re v for the coefficients c' whose columns
-N1/2 < m < 0 are, off the Nyquist row, the conjugate mirrors of the columns
-m (the Nyquist row and column evaluated literally).  For the Hermitian
coefficients of real fields c' = c.
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


def run(torch, coeffs, lon, colat, n_lon, n_lat, dtype, tol, options=None):
    from paper_2605_01313_gb300 import Plan
    cd = torch.complex128 if dtype == "f64" else torch.complex64
    with Plan(n_lon, n_lat, tol, dtype, coeffs.shape[0], options=options) as plan:
        plan.set_points(torch.from_numpy(np.ascontiguousarray(lon)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(colat)).cuda())
        out = plan.execute(torch.from_numpy(coeffs).to(cd).cuda())
        torch.cuda.synchronize()
        params = plan.params
        return out.cpu().numpy(), params


def mirror_substituted(c):
    """c' of a real-field plan: in the columns -N1/2 < m < 0, every entry off
    the Nyquist row replaced by conj(c_{-n,-m}); the Nyquist row and column
    kept as they are."""
    F, N2, N1 = c.shape
    h1 = N1 // 2
    out = c.copy()
    for q in range(1, h1):                  # m = q - h1 in (-h1, 0)
        qm = N1 - q                         # column of -m
        for r in range(1, N2):              # n = r - N2/2 > -N2/2; -n at row N2 - r
            out[:, r, q] = np.conj(c[:, N2 - r, qm])
    return out


def max_rel_err(vals, coeffs, lon, colat):
    ref = oracle.evaluate(coeffs, lon, colat)
    return max(oracle.rel_linf(vals[f], ref[f].real) for f in range(coeffs.shape[0]))


def real_opts(**kw):
    from paper_2605_01313_gb300.nufft import Options
    return Options.make(real_fields=True, **kw)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_real_fields_c2(torch_cuda, dtype):
    wl = synth.workload_c2(dtype)
    s = wl.sample
    vals, prm = run(torch_cuda, wl.coeffs, wl.lon, wl.colat, wl.n_lon, wl.n_lat, dtype, wl.tol,
                    real_opts())
    assert prm["flags"] == 1
    err = max_rel_err(vals[:, s], wl.coeffs, wl.lon[s], wl.colat[s])
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


def test_real_fields_c3_f32_full_size(torch_cuda):
    wl = synth.workload_c3("f32")
    s = wl.sample
    vals, _ = run(torch_cuda, wl.coeffs, wl.lon, wl.colat, wl.n_lon, wl.n_lat, "f32", wl.tol,
                  real_opts())
    assert np.all(np.isfinite(vals))
    assert max_rel_err(vals[:, s], wl.coeffs, wl.lon[s], wl.colat[s]) <= TOL_F32


@pytest.mark.parametrize("n_lon,n_lat", [(8, 4), (6, 5), (10, 6), (22, 11), (64, 32),
                                         (96, 48), (256, 128)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_real_fields_nyquist_and_non_hermitian(torch_cuda, n_lon, n_lat, dtype):
    """Arbitrary complex coefficients (not Hermitian, Nyquist row and column
    non-zero): the real-field plan gives Re v of the mirror-substituted
    coefficients.  Odd N1/2 (n_lon = 6, 10, 22) takes the plain-load theta pass."""
    rng = np.random.default_rng(300 + n_lon + n_lat)
    F, N2, N1 = 2, 2 * n_lat, n_lon
    c = (rng.standard_normal((F, N2, N1)) + 1j * rng.standard_normal((F, N2, N1))) / (N1 * N2)
    P = 1500
    lon = rng.uniform(-1.0, 2 * math.pi + 1.0, P)
    colat = rng.uniform(-math.pi, math.pi, P)
    tol = 1e-12 if dtype == "f64" else 1e-6
    vals, _ = run(torch_cuda, c, lon, colat, n_lon, n_lat, dtype, tol, real_opts())
    # scale by the largest coefficient magnitude: c' is arbitrary, not smooth
    ref = oracle.evaluate(mirror_substituted(c), lon, colat)
    bound = (TOL_F64 if dtype == "f64" else TOL_F32)
    for f in range(F):
        scale = np.abs(c[f]).sum()
        err = np.max(np.abs(vals[f] - ref[f].real)) / scale
        assert err <= bound, (f, err)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_real_fields_match_general_plan_on_hermitian_input(torch_cuda, dtype):
    wl = synth.small_workload(77, 128, 64, n_fields=3, dtype=dtype, points="divergent")
    # make the Nyquist row and column non-zero as well (evaluated literally by both)
    rng = np.random.default_rng(77)
    c = wl.coeffs.copy()
    c[:, 0, :] += 1e-3 * (rng.standard_normal(c[:, 0, :].shape)
                          + 1j * rng.standard_normal(c[:, 0, :].shape))
    c[:, :, 0] += 1e-3 * (rng.standard_normal(c[:, :, 0].shape)
                          + 1j * rng.standard_normal(c[:, :, 0].shape))
    general, _ = run(torch_cuda, c, wl.lon, wl.colat, 128, 64, dtype, wl.tol)
    real, _ = run(torch_cuda, c, wl.lon, wl.colat, 128, 64, dtype, wl.tol, real_opts())
    scale = np.max(np.abs(general))
    assert np.max(np.abs(general - real)) / scale <= (TOL_F64 if dtype == "f64" else TOL_F32)
    assert max_rel_err(real, c, wl.lon, wl.colat) <= (TOL_F64 if dtype == "f64" else TOL_F32)


@pytest.mark.parametrize("dtype,tol,bound", [("f64", 1e-12, TOL_F64), ("f64", 1e-9, 1e-8),
                                             ("f32", 1e-6, TOL_F32), ("f64", 1e-6, 1e-5)])
def test_sigma4(torch_cuda, dtype, tol, bound):
    from paper_2605_01313_gb300.nufft import Options
    wl = synth.small_workload(55, 256, 128, n_fields=2, dtype=dtype, points="uniform", tol=tol)
    vals, prm = run(torch_cuda, wl.coeffs, wl.lon, wl.colat, 256, 128, dtype, tol,
                    Options.make(sigma=4))
    assert prm["sigma"] == 4 and prm["n1"] == 1024 and prm["n2"] == 1024
    assert max_rel_err(vals, wl.coeffs, wl.lon, wl.colat) <= bound


@pytest.mark.parametrize("tile", [(8, 8), (16, 32), (64, 16), (128, 64), (32, 128)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_bin_sizes(torch_cuda, tile, dtype):
    from paper_2605_01313_gb300.nufft import Options
    wl = synth.small_workload(56, 512, 256, n_fields=3, dtype=dtype, points="divergent")
    vals, prm = run(torch_cuda, wl.coeffs, wl.lon, wl.colat, 512, 256, dtype, wl.tol,
                    Options.make(tile=tile, real_fields=True))
    assert (prm["tile_x"], prm["tile_y"]) == tile
    s = np.arange(0, wl.lon.size, 37)
    err = max_rel_err(vals[:, s], wl.coeffs, wl.lon[s], wl.colat[s])
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


def test_wider_kernel_is_at_least_as_accurate(torch_cuda):
    from paper_2605_01313_gb300.nufft import Options
    wl = synth.small_workload(57, 128, 64, n_fields=1, dtype="f64", points="uniform", tol=1e-6)
    errs = []
    for w in (5, 7, 9):
        vals, prm = run(torch_cuda, wl.coeffs, wl.lon, wl.colat, 128, 64, "f64", 1e-6,
                        Options.make(w=w))
        assert prm["w"] == w
        errs.append(max_rel_err(vals, wl.coeffs, wl.lon, wl.colat))
    assert errs[0] > errs[1] > errs[2], errs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("points", ["divergent", "uniform"])
@pytest.mark.parametrize("real", [False, True])
def test_keep_order_points(torch_cuda, dtype, points, real):
    """Unsorted evaluation in the caller's order gives the oracle's values for
    grid-ordered departure points and for scattered points alike."""
    from paper_2605_01313_gb300.nufft import Options
    wl = synth.small_workload(81, 256, 128, n_fields=3, dtype=dtype, points=points)
    vals, prm = run(torch_cuda, wl.coeffs, wl.lon, wl.colat, 256, 128, dtype, wl.tol,
                    Options.make(keep_order=True, real_fields=real))
    assert prm["flags"] & 2
    s = np.arange(0, wl.lon.size, 11)
    err = max_rel_err(vals[:, s], wl.coeffs, wl.lon[s], wl.colat[s])
    assert err <= (TOL_F64 if dtype == "f64" else TOL_F32), err


def test_keep_order_batched_and_seams(torch_cuda):
    """Batched members with different point counts, points on both seams of the torus."""
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.nufft import Options
    torch = torch_cuda
    rng = np.random.default_rng(82)
    wls = [synth.workload_member(950 + k, 128, 64, "f32", n_sample=300) for k in range(3)]
    pts = [(w.lon.copy(), w.colat.copy()) for w in wls]
    pts[1][0][:50] = rng.uniform(-1e-4, 1e-4, 50)
    pts[1][1][:50] = rng.uniform(-1e-4, 1e-4, 50)
    pts[2][1][:30] = math.pi + rng.uniform(-1e-4, 1e-4, 30)
    pts[2] = (pts[2][0][:4000], pts[2][1][:4000])          # a shorter member
    lon = torch.from_numpy(np.concatenate([p[0] for p in pts])).cuda()
    colat = torch.from_numpy(np.concatenate([p[1] for p in pts])).cuda()
    coef = torch.from_numpy(np.stack([w.coeffs for w in wls])).to(torch.complex64).cuda()
    counts = [p[0].size for p in pts]
    with Plan(128, 64, 1e-6, "f32", 3, n_members=3,
              options=Options.make(keep_order=True, real_fields=True)) as plan:
        plan.set_points(lon, colat, counts)
        outs = [o.cpu().numpy() for o in plan.split_values(plan.execute(coef))]
    for w, (plon, pcolat), o in zip(wls, pts, outs):
        s = np.concatenate([np.arange(50), w.sample[w.sample < plon.size]])
        ref = oracle.evaluate(w.coeffs, plon[s], pcolat[s])
        err = max(oracle.rel_linf(o[f][s], ref[f].real) for f in range(3))
        assert err <= TOL_F32, err
