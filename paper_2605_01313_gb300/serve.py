"""Python side of the serving engine (csrc/serve.cu): a thin wrapper of the
dfsnufft_server C ABI, plus a Poisson load generator used by the benchmark."""
from __future__ import annotations

import ctypes
import threading
import time

import numpy as np

from . import nufft


class Server:
    """Continuous-batching server (see include/dfsnufft.h).  Requests carry CUDA
    tensors: lon, colat (float64, P), coeffs (F, 2 n_lat, n_lon complex), values
    (F, P real); the tensors are kept alive until the request completes."""

    def __init__(self, tol=1e-6, dtype="f32", n_fields=3, hbm_budget=120 << 30, max_batch=8,
                 options=None):
        self.dtype = dtype
        self.n_fields = int(n_fields)
        h = ctypes.c_void_p()
        nufft._check(nufft.lib().dfsnufft_server_create_opts(
            float(tol), nufft._dtype_code(dtype), self.n_fields, int(hbm_budget), int(max_batch),
            ctypes.byref(options) if options is not None else None, ctypes.byref(h)))
        self._h = h
        self._live = {}
        self._lock = threading.Lock()

    def submit(self, n_lon, n_lat, lon, colat, coeffs, values):
        r = nufft.Request(int(n_lon), int(n_lat), int(lon.numel()), lon.data_ptr(),
                          colat.data_ptr(), coeffs.data_ptr(), values.data_ptr())
        t = ctypes.c_int64()
        nufft._check(nufft.lib().dfsnufft_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        with self._lock:
            self._live[t.value] = (lon, colat, coeffs, values)
        return t.value

    def wait(self, ticket, timeout=60.0):
        st = ctypes.c_int()
        lat = ctypes.c_double()
        rc = nufft.lib().dfsnufft_server_wait(self._h, int(ticket), float(timeout),
                                              ctypes.byref(st), ctypes.byref(lat))
        if rc != nufft.OK:
            raise nufft.DfsError(rc, "waiting for request %d" % ticket)
        with self._lock:
            self._live.pop(ticket, None)
        return st.value, lat.value

    def stats(self):
        s = nufft.ServerStats()
        nufft._check(nufft.lib().dfsnufft_server_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nufft.lib().dfsnufft_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_run(server, requests, rate, duration, seed=0):
    """Submit requests drawn round-robin from ``requests`` (dicts with keys
    n_lon, n_lat, lon, colat, coeffs, values, pf = points x fields) at Poisson
    arrival ``rate`` (1/s) for ``duration`` seconds and wait for all of them.
    Returns the latencies (s, measured by the server from submit to
    completion), the point-fields done, the wall time from the first submit to
    the last completion, and the number of requests."""
    import queue
    rng = np.random.default_rng(seed)
    tickets = queue.Queue()
    errors, lat = [], []
    pf_done = [0]

    def waiter():
        while True:
            item = tickets.get()
            if item is None:
                return
            tk, pf = item
            try:
                st, l = server.wait(tk, timeout=max(60.0, 10 * duration))
            except Exception as e:      # noqa: BLE001 - reported below
                errors.append(repr(e))
                continue
            if st != 0:
                errors.append("status %d" % st)
            lat.append(l)
            pf_done[0] += pf

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    t0 = time.perf_counter()
    t_next = 0.0
    n = 0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next > duration:
            break
        now = time.perf_counter() - t0
        if t_next > now:
            time.sleep(t_next - now)
        req = requests[n % len(requests)]
        n += 1
        tk = server.submit(req["n_lon"], req["n_lat"], req["lon"], req["colat"], req["coeffs"],
                           req["values"])
        tickets.put((tk, req["pf"]))
    tickets.put(None)
    th.join()
    wall = time.perf_counter() - t0
    if errors:
        raise RuntimeError("serving errors: %s" % errors[:3])
    return np.array(lat), pf_done[0], wall, n
