"""Failure detection without a GPU fault: a bounded wait that nothing
completes gives up, reports the timeout through the device status word, and
leaves the context usable."""
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


def test_bounded_wait_times_out_and_context_survives(torch_cuda):
    from paper_2605_01313_gb300 import nufft, Plan
    status, ms = nufft.dfsnufft_selftest_wait_timeout(200_000_000)   # ~0.1 s of SM cycles
    assert status == 1
    assert ms > 20.0, ms                   # it waited before giving up
    # the same process keeps computing correctly afterwards
    wl = synth.small_workload(5, 64, 32, n_fields=2, dtype="f64")
    torch = torch_cuda
    with Plan(64, 32, wl.tol, "f64", 2) as plan:
        plan.set_points(torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda())
        vals = plan.execute(torch.from_numpy(wl.coeffs).cuda()).cpu().numpy()
        plan.check()
    ref = oracle.evaluate(wl.coeffs, wl.lon, wl.colat)
    assert max(oracle.rel_linf(vals[f], ref[f].real) for f in range(2)) <= 1e-11


def test_selftest_rejects_unbounded_budget(torch_cuda):
    from paper_2605_01313_gb300 import nufft
    for bad in (0, -5, 5_000_000_000):
        with pytest.raises(nufft.DfsError) as ei:
            nufft.dfsnufft_selftest_wait_timeout(bad)
        assert ei.value.status == nufft.ERR_INVALID_ARG
