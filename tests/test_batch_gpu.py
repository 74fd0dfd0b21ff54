"""Batched plans (members of one grid, each with its own points) and ensembles on
uneven grids (one CUDA graph per step) against single-member plans and the
oracle."""
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


def _single(torch, wl):
    from paper_2605_01313_gb300 import Plan
    cd = torch.complex128 if wl.dtype == "f64" else torch.complex64
    with Plan(wl.n_lon, wl.n_lat, wl.tol, wl.dtype, wl.n_fields) as plan:
        plan.set_points(torch.from_numpy(wl.lon).cuda(), torch.from_numpy(wl.colat).cuda())
        out = plan.execute(torch.from_numpy(wl.coeffs).to(cd).cuda())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def _members(n, n_lon, n_lat, dtype, seed0, ragged=True):
    wls = []
    rng = np.random.default_rng(seed0)
    for k in range(n):
        wl = synth.workload_member(seed0 + k, n_lon, n_lat, dtype, n_sample=64)
        if ragged and k % 2:
            keep = np.sort(rng.choice(wl.n_points, wl.n_points - 37 * k, replace=False))
            wl = synth.Workload(wl.name, n_lon, n_lat, wl.coeffs, wl.lon[keep], wl.colat[keep],
                                wl.tol, dtype, sample=np.arange(0, keep.size, 7))
        wls.append(wl)
    return wls


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_plan_equals_single_plans(torch_cuda, dtype):
    from paper_2605_01313_gb300 import Plan
    torch = torch_cuda
    wls = _members(5, 128, 64, dtype, 500)
    cd = torch.complex128 if dtype == "f64" else torch.complex64
    coeffs = torch.from_numpy(np.stack([w.coeffs for w in wls])).to(cd).cuda()
    lon = torch.from_numpy(np.concatenate([w.lon for w in wls])).cuda()
    colat = torch.from_numpy(np.concatenate([w.colat for w in wls])).cuda()
    counts = [w.n_points for w in wls]
    with Plan(128, 64, wls[0].tol, dtype, 3, n_members=len(wls)) as plan:
        plan.set_points(lon, colat, counts)
        out = plan.execute(coeffs)
        torch.cuda.synchronize()
        views = [v.cpu().numpy() for v in plan.split_values(out)]
    bound = 1e-11 if dtype == "f64" else 2e-5
    for wl, got in zip(wls, views):
        assert np.array_equal(got, _single(torch, wl))
        ref = oracle.evaluate(wl.coeffs, wl.lon[wl.sample], wl.colat[wl.sample])
        for f in range(3):
            assert oracle.rel_linf(got[f][wl.sample], ref[f].real) <= bound


def _check_members_against_oracle(wls, vals, bound=2e-5):
    off = 0
    for wl in wls:
        got = vals[off:off + 3 * wl.n_points].reshape(3, wl.n_points)
        off += 3 * wl.n_points
        ref = oracle.evaluate(wl.coeffs, wl.lon[wl.sample], wl.colat[wl.sample])
        for f in range(3):
            assert oracle.rel_linf(got[f][wl.sample], ref[f].real) <= bound, (wl.name, f)


def test_ensemble_graph_uneven_grids(torch_cuda):
    """Groups of 128x64, 256x128, 512x256 and 1024x512 members (the ensemble's
    grid sizes) in one graph: every member within 2e-5 of the oracle at its
    seeded sample points; replays give the same values, and new points
    re-record the graph."""
    torch = torch_cuda
    groups = [(3, 128, 64), (2, 256, 128), (2, 512, 256), (1, 1024, 512)]
    ens = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3)
    all_wls, pts, cfs, outs = [], [], [], []
    for gi, (m, n_lon, n_lat) in enumerate(groups):
        wls = _members(m, n_lon, n_lat, "f32", 700 + 10 * gi)
        all_wls.append(wls)
        pts.append((torch.from_numpy(np.concatenate([w.lon for w in wls])).cuda(),
                    torch.from_numpy(np.concatenate([w.colat for w in wls])).cuda(),
                    [w.n_points for w in wls]))
        cfs.append(torch.from_numpy(np.stack([w.coeffs for w in wls])).to(torch.complex64).cuda())
        outs.append(torch.zeros(3 * sum(w.n_points for w in wls), dtype=torch.float32,
                                device="cuda"))
    ens.run(pts, cfs, outs)          # runs, then records
    ens.check()
    first = [o.cpu().numpy().copy() for o in outs]
    for wls, vals in zip(all_wls, first):
        _check_members_against_oracle(wls, vals)
    for o in outs:
        o.zero_()
    ens.run(pts, cfs, outs)          # graph replay
    ens.check()
    for a, o in zip(first, outs):
        assert np.array_equal(a, o.cpu().numpy())
    for wls, vals in zip(all_wls, first):
        off = 0
        for wl in wls:
            got = vals[off:off + 3 * wl.n_points].reshape(3, wl.n_points)
            off += 3 * wl.n_points
            assert np.array_equal(got, _single(torch, wl))
    # other points for the first group: the graph is recorded again
    wl2 = _members(3, 128, 64, "f32", 900, ragged=False)
    pts[0] = (torch.from_numpy(np.concatenate([w.lon for w in wl2])).cuda(),
              torch.from_numpy(np.concatenate([w.colat for w in wl2])).cuda(),
              [w.n_points for w in wl2])
    cfs[0] = torch.from_numpy(np.stack([w.coeffs for w in wl2])).to(torch.complex64).cuda()
    outs[0] = torch.zeros(3 * sum(w.n_points for w in wl2), dtype=torch.float32, device="cuda")
    ens.run(pts, cfs, outs)
    ens.check()
    vals = outs[0].cpu().numpy()
    _check_members_against_oracle(wl2, vals)
    off = 0
    for wl in wl2:
        got = vals[off:off + 3 * wl.n_points].reshape(3, wl.n_points)
        off += 3 * wl.n_points
        assert np.array_equal(got, _single(torch, wl))
    ens.destroy()


def _ensemble_inputs(torch, groups, seed0, real=False):
    all_wls, pts, cfs, outs = [], [], [], []
    for gi, (m, n_lon, n_lat) in enumerate(groups):
        wls = _members(m, n_lon, n_lat, "f32", seed0 + 10 * gi)
        all_wls.append(wls)
        pts.append((torch.from_numpy(np.concatenate([w.lon for w in wls])).cuda(),
                    torch.from_numpy(np.concatenate([w.colat for w in wls])).cuda(),
                    [w.n_points for w in wls]))
        cfs.append(torch.from_numpy(np.stack([w.coeffs for w in wls])).to(torch.complex64).cuda())
        outs.append(torch.zeros(3 * sum(w.n_points for w in wls), dtype=torch.float32,
                                device="cuda"))
    return all_wls, pts, cfs, outs


@pytest.mark.parametrize("real", [False, True])
def test_ensemble_persistent_launch(torch_cuda, real):
    """The persistent step (one launch draining every group's theta, phi and
    interpolation tasks) gives every member within 2e-5 of the oracle and of
    the fork/join graph, and the same values on a graph replay."""
    torch = torch_cuda
    groups = [(3, 128, 64), (2, 256, 128), (2, 512, 256), (1, 1024, 512)]
    opts = [nufft.Options.make(real_fields=real) for _ in groups]
    all_wls, pts, cfs, outs = _ensemble_inputs(torch, groups, 1100)
    ref_outs = [torch.zeros_like(o) for o in outs]
    forkjoin = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3, options=opts)
    forkjoin.run(pts, cfs, ref_outs)
    forkjoin.check()
    ens = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3, options=opts,
                         persistent=True)
    ens.run(pts, cfs, outs)            # runs, then records
    ens.check()
    first = [o.cpu().numpy().copy() for o in outs]
    for wls, vals, ref in zip(all_wls, first, ref_outs):
        _check_members_against_oracle(wls, vals)
        r = ref.cpu().numpy()
        assert np.max(np.abs(vals - r)) <= 2e-5 * np.max(np.abs(r))
    for o in outs:
        o.zero_()
    ens.run(pts, cfs, outs)            # graph replay
    ens.check()
    for a, o in zip(first, outs):
        assert np.array_equal(a, o.cpu().numpy())
    ens.destroy()
    forkjoin.destroy()


def test_ensemble_persistent_queue_wait_times_out(torch_cuda):
    """A queue wait that can never complete gives up after its cycle budget,
    the step reports DFSNUFFT_ERR_TIMEOUT, and the next step computes
    correctly (failure detection without a GPU fault)."""
    torch = torch_cuda
    groups = [(2, 128, 64), (1, 256, 128)]
    all_wls, pts, cfs, outs = _ensemble_inputs(torch, groups, 1200)
    ens = nufft.Ensemble(groups, tol=1e-6, dtype="f32", n_fields=3, persistent=True)
    ens.run(pts, cfs, outs)
    ens.check()
    assert ens.selftest_queue_timeout(2_000_000) == nufft.ERR_TIMEOUT   # ~1 ms of SM cycles
    for o in outs:
        o.zero_()
    ens.run(pts, cfs, outs)
    ens.check()
    for wls, o in zip(all_wls, outs):
        _check_members_against_oracle(wls, o.cpu().numpy())
    ens.destroy()


def test_ensemble_persistent_unsupported_kinds(torch_cuda):
    """FP64 ensembles and unsorted points keep the fork/join form."""
    with pytest.raises(nufft.DfsError) as ei:
        nufft.Ensemble([(1, 128, 64)], tol=1e-12, dtype="f64", n_fields=3, persistent=True)
    assert ei.value.status == nufft.ERR_UNSUPPORTED
    with pytest.raises(nufft.DfsError) as ei:
        nufft.Ensemble([(1, 128, 64)], tol=1e-6, dtype="f32", n_fields=3, persistent=True,
                       options=[nufft.Options.make(keep_order=True)])
    assert ei.value.status == nufft.ERR_UNSUPPORTED
