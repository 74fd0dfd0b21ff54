"""The serving engine: results are the same alone and in a mix of concurrent
requests, admission respects the HBM budget, and requests that can never fit
are refused rather than left waiting."""
import threading

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


def _request(torch, seed, n_lon, n_lat):
    wl = synth.workload_member(seed, n_lon, n_lat, "f32", n_sample=48)
    return {"wl": wl, "n_lon": n_lon, "n_lat": n_lat,
            "lon": torch.from_numpy(wl.lon).cuda(), "colat": torch.from_numpy(wl.colat).cuda(),
            "coeffs": torch.from_numpy(wl.coeffs).to(torch.complex64).cuda(),
            "values": torch.full((3, wl.n_points), float("nan"), dtype=torch.float32,
                                 device="cuda")}


def _submit(srv, r):
    return srv.submit(r["n_lon"], r["n_lat"], r["lon"], r["colat"], r["coeffs"], r["values"])


def test_same_alone_and_in_the_mix(torch_cuda):
    from paper_2605_01313_gb300 import Plan
    from paper_2605_01313_gb300.serve import Server
    torch = torch_cuda
    sizes = [(128, 64), (256, 128), (512, 256)]
    srv = Server(tol=1e-6, dtype="f32", n_fields=3, hbm_budget=8 << 30, max_batch=4)
    target = _request(torch, 4242, 256, 128)
    st, _ = srv.wait(_submit(srv, target))
    assert st == 0
    alone = target["values"].cpu().numpy().copy()
    # the same request inside a burst of mixed requests
    mix = [_request(torch, 5000 + i, *sizes[i % 3]) for i in range(24)]
    target["values"].fill_(float("nan"))
    tickets = [_submit(srv, r) for r in mix[:12]]
    tickets.append(_submit(srv, target))
    tickets += [_submit(srv, r) for r in mix[12:]]
    for tk in tickets:
        st, lat = srv.wait(tk)
        assert st == 0 and lat > 0
    assert np.array_equal(target["values"].cpu().numpy(), alone)
    stats = srv.stats()
    assert stats["batches"] < stats["completed"]          # some requests shared a launch
    # each served result equals a plain plan's and the oracle's
    for r in mix[:6] + [target]:
        wl = r["wl"]
        got = r["values"].cpu().numpy()
        with Plan(wl.n_lon, wl.n_lat, 1e-6, "f32", 3) as plan:
            plan.set_points(r["lon"], r["colat"])
            ref = plan.execute(r["coeffs"]).cpu().numpy()
        assert np.array_equal(got, ref)
        o = oracle.evaluate(wl.coeffs, wl.lon[wl.sample], wl.colat[wl.sample])
        for f in range(3):
            assert oracle.rel_linf(got[f][wl.sample], o[f].real) <= 2e-5
    srv.close()


def test_budget_admission_and_refusal(torch_cuda):
    from paper_2605_01313_gb300.serve import Server
    torch = torch_cuda
    # room for one 256x128 slot of two members (about 23 MB): requests queue and
    # run one batch at a time
    srv = Server(tol=1e-6, dtype="f32", n_fields=3, hbm_budget=40 << 20, max_batch=2)
    reqs = [_request(torch, 6000 + i, 256, 128) for i in range(6)]
    tickets = [_submit(srv, r) for r in reqs]
    for tk in tickets:
        st, _ = srv.wait(tk)
        assert st == 0
    s = srv.stats()
    assert s["slots"] == 1 and s["reserved_bytes"] <= s["budget_bytes"]
    # a 1024x512 request needs far more than the budget: refused, not stuck
    big = _request(torch, 6100, 1024, 512)
    st, _ = srv.wait(_submit(srv, big))
    assert st == nufft.ERR_OOM
    # the server keeps serving afterwards
    st, _ = srv.wait(_submit(srv, reqs[0]))
    assert st == 0
    srv.close()


def test_concurrent_submitters(torch_cuda):
    from paper_2605_01313_gb300.serve import Server
    torch = torch_cuda
    srv = Server(tol=1e-6, dtype="f32", n_fields=3, hbm_budget=4 << 30, max_batch=8)
    reqs = [_request(torch, 7000 + i, *((128, 64) if i % 2 else (256, 128))) for i in range(16)]
    results = {}

    def client(chunk):
        for r in chunk:
            results[id(r)] = srv.wait(_submit(srv, r))[0]

    threads = [threading.Thread(target=client, args=(reqs[i::4],)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert len(results) == 16 and all(v == 0 for v in results.values())
    for r in reqs:
        assert np.all(np.isfinite(r["values"].cpu().numpy()))
    srv.close()
