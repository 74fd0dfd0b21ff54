"""The autotuner (dfsnufft_autotune) on the GPU: its choice is accurate
against the FP64 oracle, no slower than the default, and cached."""
import json
import os
import time

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


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_tune_small_batch(torch_cuda, tmp_path, dtype):
    from paper_2605_01313_gb300 import autotune, Plan
    torch = torch_cuda
    tol = 1e-6 if dtype == "f32" else 1e-12
    cd = torch.complex64 if dtype == "f32" else torch.complex128
    wls = [synth.workload_member(900 + k, 256, 128, dtype, n_sample=200) for k in range(3)]
    lon = torch.from_numpy(np.concatenate([w.lon for w in wls])).cuda()
    colat = torch.from_numpy(np.concatenate([w.colat for w in wls])).cuda()
    coef = torch.from_numpy(np.stack([w.coeffs for w in wls])).to(cd).cuda()
    counts = [w.n_points for w in wls]
    cache = str(tmp_path / "tune.json")
    best, cands = autotune.tune(256, 128, lon, colat, counts, coef, tol=tol, dtype=dtype,
                                n_fields=3, path=cache)
    ok = [c for c in cands if c["status"] == 0]
    assert len(ok) >= 10
    bound = (20 if dtype == "f32" else 10) * tol
    chosen = [c for c in ok if c["opts"] == best.as_dict()]
    assert len(chosen) == 1 and chosen[0]["err"] <= bound
    default = [c for c in ok if c["opts"]["tile_x"] == 0 and c["opts"]["w"] == 0
               and c["opts"]["sigma"] == 0]
    assert default and chosen[0]["ms"] <= default[0]["ms"] * 1.0001
    # every accepted candidate's error really is within the bound: check the
    # chosen one against the oracle on member 1
    with Plan(256, 128, tol, dtype, 3, n_members=3, options=best) as plan:
        plan.set_points(lon, colat, counts)
        out = plan.split_values(plan.execute(coef))[1].cpu().numpy()
    w1 = wls[1]
    ref = oracle.evaluate(w1.coeffs, w1.lon[w1.sample], w1.colat[w1.sample])
    err = max(oracle.rel_linf(out[f][w1.sample], ref[f].real) for f in range(3))
    assert err <= bound, err
    # cached: the same key returns at once with the same choice
    table = json.load(open(cache))
    assert len(table) == 1
    t0 = time.perf_counter()
    best2, _ = autotune.tune(256, 128, lon, colat, counts, coef, tol=tol, dtype=dtype,
                             n_fields=3, path=cache)
    assert time.perf_counter() - t0 < 0.5
    assert best2.as_dict() == best.as_dict()


def test_tune_rejects_bad_args(torch_cuda):
    from paper_2605_01313_gb300 import nufft
    import ctypes
    a = nufft.TuneArgs()
    best = nufft.Options()
    n = ctypes.c_int()
    rc = nufft.lib().dfsnufft_autotune(ctypes.byref(a), None, 0, ctypes.byref(n),
                                       ctypes.byref(best))
    assert rc == nufft.ERR_INVALID_ARG
