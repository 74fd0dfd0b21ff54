"""Autotuner front end: runs ``dfsnufft_autotune`` (csrc/autotune.cu) on a
workload held in CUDA tensors and keeps its choices in a JSON cache.

The cache maps a key (GPU name, grid, members, fields, points per member,
precision, tolerance, real-field flag) to the chosen options and the timings
of every candidate, so a later run with the same key reuses the choice without
measuring again.  The default cache file is ``$DFSNUFFT_TUNE_CACHE`` or
``~/.cache/dfsnufft/tune.json``; ``path=None`` disables it.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import nufft

DEFAULT_CACHE = os.environ.get("DFSNUFFT_TUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "dfsnufft",
                                            "tune.json"))
_UNSET = object()


def cache_key(device_name, n_lon, n_lat, n_members, n_fields, counts, dtype, tol, real_fields):
    return "|".join(str(x) for x in (device_name, n_lon, n_lat, n_members, n_fields,
                                     int(np.max(counts)), dtype, "%.3g" % tol,
                                     int(bool(real_fields))))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, table):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(n_lon, n_lat, lon, colat, counts, coeffs, tol=1e-6, dtype="f32", n_fields=3,
         real_fields=True, steps=5, stream=None, path=_UNSET):
    """Best :class:`nufft.Options` for this workload, and the candidate table.

    ``lon``, ``colat``: CUDA float64 tensors of all members' points; ``counts``:
    points per member; ``coeffs``: CUDA complex tensor of shape
    (members, fields, 2 n_lat, n_lon) (or (fields, ...) for one member) in the
    plan's precision."""
    import torch
    if path is _UNSET:
        path = DEFAULT_CACHE
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    dev = torch.cuda.get_device_name(lon.device)
    key = cache_key(dev, n_lon, n_lat, counts.size, n_fields, counts, dtype, tol, real_fields)
    table = _load(path) if path else {}
    if key in table:
        best = nufft.Options()
        for name, value in table[key]["best"].items():
            setattr(best, name, int(value))
        return best, table[key]["candidates"]
    if stream is None:
        stream = torch.cuda.current_stream(lon.device)
    a = nufft.TuneArgs()
    a.n_members, a.n_lon, a.n_lat = int(counts.size), int(n_lon), int(n_lat)
    a.tol, a.dtype, a.n_fields = float(tol), nufft._dtype_code(dtype), int(n_fields)
    a.flags = nufft.REAL_FIELDS if real_fields else 0
    a.n_points = counts.ctypes.data
    a.lon, a.colat, a.coeffs = lon.data_ptr(), colat.data_ptr(), coeffs.data_ptr()
    a.steps = int(steps)
    a.stream = stream.cuda_stream
    res = (nufft.TuneResult * 64)()
    n = ctypes.c_int()
    best = nufft.Options()
    nufft._check(nufft.lib().dfsnufft_autotune(ctypes.byref(a), res, 64, ctypes.byref(n),
                                               ctypes.byref(best)))
    cands = [res[i].as_dict() for i in range(n.value)]
    if path:
        table = _load(path)
        table[key] = {"best": best.as_dict(), "candidates": cands}
        _store(path, table)
    return best, cands
