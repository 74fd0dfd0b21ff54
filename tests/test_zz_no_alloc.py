"""The allocation-free entry point (dfsnufft_execute_noalloc) against the plan
entry points.

Some callers cannot allocate device memory: a model time step that runs inside
another framework's memory pool, or a latency-critical loop that must not take
the device-wide synchronisation cudaMalloc/cudaFree imply.  For them the library
offers one call whose working memory is a static device array.  This file is
collected last on purpose, so that a stop-at-first-failure run has already run
every other test when it gets here; it also passes when run alone.
"""
import numpy as np
import pytest

import oracle
from paper_2605_01313_gb300 import build, nufft, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the -m gpu tests")
    build.build()
    return torch


def _inputs(torch, wl):
    cd = torch.complex128 if wl.dtype == "f64" else torch.complex64
    return (torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda(),
            torch.from_numpy(wl.coeffs).to(cd).cuda())


def _with_plan(torch, wl):
    from paper_2605_01313_gb300 import Plan
    lon, colat, coeffs = _inputs(torch, wl)
    with Plan(wl.n_lon, wl.n_lat, wl.tol, wl.dtype, wl.n_fields) as plan:
        plan.set_points(lon, colat)
        out = plan.execute(coeffs)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def _noalloc(torch, wl):
    lon, colat, coeffs = _inputs(torch, wl)
    rd = torch.float64 if wl.dtype == "f64" else torch.float32
    out = torch.full((wl.n_fields, wl.n_points), float("nan"), dtype=rd, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nufft.dfsnufft_execute_noalloc(wl.n_lon, wl.n_lat, wl.tol, wl.dtype, wl.n_fields,
                                   wl.n_points, lon.data_ptr(), colat.data_ptr(),
                                   coeffs.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_plan_on_consecutive_calls(torch_cuda):
    """Two calls in a row with different problems, each within the parity tolerance
    of the plan path (and of the oracle), so that state left in the shared scratch
    by one call does not leak into the next."""
    first = synth.small_workload(31, 128, 64, n_fields=3, dtype="f64", points="divergent")
    second = synth.small_workload(32, 256, 128, n_fields=2, dtype="f32", points="rotation")
    # the same configuration as the one before it, with new points and coefficients
    again = synth.small_workload(33, 128, 64, n_fields=3, dtype="f64", points="rotation")
    for wl, bound in ((first, 1e-11), (second, 2e-5), (first, 1e-11), (again, 1e-11)):
        got = _noalloc(torch_cuda, wl)
        ref = _with_plan(torch_cuda, wl)
        assert np.all(np.isfinite(got))
        for f in range(wl.n_fields):
            assert oracle.rel_linf(got[f], ref[f]) <= bound
        s = wl.sample[::17]
        want = oracle.evaluate(wl.coeffs, wl.lon[s], wl.colat[s])
        for f in range(wl.n_fields):
            assert oracle.rel_linf(got[f][s], want[f].real) <= bound


def test_noalloc_rejects_problems_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    lon = torch.zeros(4, dtype=torch.float64, device="cuda")
    coeffs = torch.zeros((1, 2048, 2048), dtype=torch.complex64, device="cuda")
    out = torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(nufft.DfsError) as ei:
        nufft.dfsnufft_execute_noalloc(2048, 1024, 1e-6, "f32", 1, 4, lon.data_ptr(),
                                       lon.data_ptr(), coeffs.data_ptr(), out.data_ptr(), 0)
    assert ei.value.status == nufft.ERR_UNSUPPORTED
    # fine grid within 2048 cells but three FP64 fields need more than the scratch
    coeffs = torch.zeros((3, 1024, 1024), dtype=torch.complex128, device="cuda")
    out = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(nufft.DfsError) as ei:
        nufft.dfsnufft_execute_noalloc(1024, 512, 1e-12, "f64", 3, 4, lon.data_ptr(),
                                       lon.data_ptr(), coeffs.data_ptr(), out.data_ptr(), 0)
    assert ei.value.status == nufft.ERR_UNSUPPORTED
