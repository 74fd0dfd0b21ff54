"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol
the header declares, and its host logic (parameters, kernel, deconvolution
factors, status strings) is right."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2605_01313_gb300 import build, nufft

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nufft.lib()


def _declared_functions():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            text = open(os.path.join(INCLUDE, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(dfsnufft_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_binding_exports():
    assert _declared_functions() == sorted(nufft.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_version(lib):
    assert "sm_103a" in nufft.dfsnufft_version()


def test_strerror_covers_every_code(lib):
    seen = set()
    for code in range(0, 8):
        s = lib.dfsnufft_strerror(code).decode()
        assert s and s != "unknown status"
        seen.add(s)
    assert len(seen) == 8
    assert lib.dfsnufft_strerror(99).decode() == "unknown status"


@pytest.mark.parametrize("tol,w,w32", [(1e-1, 2, 2), (1e-3, 5, 4), (1e-6, 7, 7), (1e-9, 11, None),
                                       (1e-12, 14, None), (1e-14, 16, None)])
def test_width_rule(lib, tol, w, w32):
    p = nufft.dfsnufft_choose_params(64, 32, tol, "f64")
    assert p["w"] == w
    assert p["beta"] == pytest.approx(2.30 * w)
    if w32 is not None:
        p = nufft.dfsnufft_choose_params(64, 32, tol, "f32")
        assert p["w"] == w32 and p["beta"] == pytest.approx(2.30 * w32)


def test_width_rule_monotone(lib):
    ws = [nufft.dfsnufft_choose_params(64, 32, 10.0 ** (-k / 4), "f64")["w"]
          for k in range(4, 57)]
    assert ws == sorted(ws) and ws[-1] == 16


def _es_band_edge_error(w, beta, n_off=201, n_freq=5):
    """Worst 1-D error of interpolating e^{i omega x} from integer samples with
    the ES kernel and exact deconvolution, over offsets x in [0, 1] and
    |omega| <= pi/2 (the band of sigma = 2): the error model of the width rule,
    computed here independently of the library's tables."""
    from scipy.integrate import quad
    def es(z):
        u = 2.0 * z / w
        out = np.zeros_like(z)
        m = np.abs(u) < 1
        out[m] = np.exp(beta * (np.sqrt(1 - u[m] ** 2) - 1))
        return out
    j = np.arange(-w, w + 2)
    x = np.linspace(0.0, 1.0, n_off)[:, None]
    worst = 0.0
    for om in np.linspace(0.0, math.pi / 2, n_freq):
        ph = 2 * quad(lambda z: math.exp(beta * (math.sqrt(1 - (2 * z / w) ** 2) - 1))
                      * math.cos(om * z), 0, w / 2, epsabs=1e-16, epsrel=1e-14, limit=400)[0]
        s = np.sum(es(x - j) * np.exp(1j * om * j), axis=1) / ph
        worst = max(worst, float(np.max(np.abs(s - np.exp(1j * om * x[:, 0])))))
    return worst


def test_width_rule_meets_corner_mode_bound(lib):
    """At tol 1e-12 the rule's width leaves a lone corner mode (1-D error in both
    dimensions) within half of the 1e-11 acceptance bound, and the next
    narrower width would not."""
    w = nufft.dfsnufft_choose_params(64, 32, 1e-12, "f64")["w"]
    e = _es_band_edge_error(w, 2.30 * w)
    e_narrow = _es_band_edge_error(w - 1, 2.30 * (w - 1))
    assert 2 * e <= 0.5e-11
    assert 2 * e_narrow > 0.5e-11


@pytest.mark.parametrize("n_lon,n_lat", [(64, 32), (160, 80), (2048, 1024), (8, 4), (24, 12)])
def test_fine_sizes(lib, n_lon, n_lat):
    p = nufft.dfsnufft_choose_params(n_lon, n_lat, 1e-12, "f64")
    assert p["N1"] == n_lon and p["N2"] == 2 * n_lat
    for n, N in ((p["n1"], p["N1"]), (p["n2"], p["N2"])):
        assert n & (n - 1) == 0 and n >= 2 * N and n >= 2 * p["w"]
        assert n < 2 * max(2 * N, 2 * p["w"], 16)


def test_parameter_errors(lib):
    bad = [((63, 32, 1e-6, "f64"), nufft.ERR_INVALID_ARG),
           ((2, 32, 1e-6, "f64"), nufft.ERR_INVALID_ARG),
           ((64, 1, 1e-6, "f64"), nufft.ERR_INVALID_ARG),
           ((64, 32, 0.0, "f64"), nufft.ERR_INVALID_ARG),
           ((64, 32, 1.5, "f64"), nufft.ERR_INVALID_ARG),
           ((64, 32, 1e-16, "f64"), nufft.ERR_TOL_UNATTAINABLE),
           ((64, 32, 5e-15, "f64"), nufft.ERR_TOL_UNATTAINABLE),
           ((64, 32, 1e-8, "f32"), nufft.ERR_TOL_UNATTAINABLE),
           ((8192, 32, 1e-6, "f32"), nufft.ERR_UNSUPPORTED),
           ((64, 4096, 1e-6, "f32"), nufft.ERR_UNSUPPORTED)]
    for args, code in bad:
        with pytest.raises(nufft.DfsError) as ei:
            nufft.dfsnufft_choose_params(*args)
        assert ei.value.status == code, args


def test_options_defaults_equal_plain_choice(lib):
    for args in ((64, 32, 1e-12, "f64"), (2048, 1024, 1e-6, "f32"), (8, 4, 1e-3, "f32")):
        a = nufft.dfsnufft_choose_params(*args)
        b = nufft.dfsnufft_choose_params(*args, options=nufft.Options())
        assert a == b
        assert a["sigma"] == 2 and a["flags"] == 0


@pytest.mark.parametrize("tol,w2,w4", [(1e-12, 14, 12), (1e-9, 11, 9), (1e-6, 7, 6),
                                       (1e-3, 5, 5), (1e-14, 16, 13)])
def test_sigma4_width_rule(lib, tol, w2, w4):
    """Oversampling 4: the narrowest width whose modelled error is at most
    that of the sigma-2 width; beta = 0.97 pi (1 - 1/8) w; fine grid 4 N."""
    p = nufft.dfsnufft_choose_params(256, 128, tol, "f64", options=nufft.Options.make(sigma=4))
    assert nufft.dfsnufft_choose_params(256, 128, tol, "f64")["w"] == w2
    assert p["w"] == w4 and p["sigma"] == 4
    assert p["beta"] == pytest.approx(0.97 * math.pi * 0.875 * w4)
    assert p["n1"] == 1024 and p["n2"] == 1024


def test_options_explicit_fields(lib):
    o = nufft.Options.make(real_fields=True, w=9, tile=(64, 8))
    p = nufft.dfsnufft_choose_params(512, 256, 1e-6, "f32", options=o)
    assert (p["w"], p["tile_x"], p["tile_y"], p["flags"]) == (9, 64, 8, 1)
    assert p["beta"] == pytest.approx(2.30 * 9)
    # at most 512 bin rows: tile_y is raised on a fine grid of 8192 rows
    p = nufft.dfsnufft_choose_params(2048, 2048, 1e-6, "f32",
                                     options=nufft.Options.make(tile=(32, 8)))
    assert p["n2"] == 8192 and p["tile_y"] == 16


@pytest.mark.parametrize("field,value", [("sigma", 3), ("sigma", 1), ("w", 1), ("w", 17),
                                         ("tile_x", 48), ("tile_x", 4), ("tile_y", 256),
                                         ("flags", 8)])
def test_options_errors(lib, field, value):
    o = nufft.Options()
    setattr(o, field, value)
    with pytest.raises(nufft.DfsError) as ei:
        nufft.dfsnufft_choose_params(64, 32, 1e-6, "f64", options=o)
    assert ei.value.status == nufft.ERR_INVALID_ARG


def test_es_kernel_shape(lib):
    w, beta = 7, 2.30 * 7
    assert nufft.dfsnufft_es_kernel(0.0, w, beta) == 1.0
    assert nufft.dfsnufft_es_kernel(3.5, w, beta) == 0.0
    assert nufft.dfsnufft_es_kernel(-3.6, w, beta) == 0.0
    for z in (0.3, 1.7, 3.2):
        a = nufft.dfsnufft_es_kernel(z, w, beta)
        assert a == nufft.dfsnufft_es_kernel(-z, w, beta)
        assert a == pytest.approx(math.exp(beta * (math.sqrt(1 - (2 * z / w) ** 2) - 1)), rel=1e-15)
    # at the edge of the support the kernel is e^{-beta}, below the tolerance it serves
    assert nufft.dfsnufft_es_kernel(3.4999999, w, beta) < 2 * math.exp(-beta) * 10


@pytest.mark.parametrize("w", [4, 7, 13])
def test_kernel_ft_against_adaptive_quadrature(lib, w):
    """Deconvolution factors (Gauss-Legendre in the library) against scipy's adaptive
    quadrature of the same integral, an independent numerical route."""
    from scipy.integrate import quad
    beta = 2.30 * w
    n_fine, n_modes = 256, 128
    ft = nufft.dfsnufft_kernel_ft(w, beta, n_fine, n_modes)
    for q in (0, 1, 17, 40, 63, 64, 100, 127):
        k = q - n_modes // 2
        xi = 2 * math.pi * k / n_fine
        f = lambda z: math.exp(beta * (math.sqrt(max(0.0, 1 - (2 * z / w) ** 2)) - 1)) * math.cos(xi * z)
        ref, _ = quad(f, -w / 2, w / 2, epsabs=1e-15, epsrel=1e-14, limit=200)
        assert ft[q] == pytest.approx(ref, rel=1e-12, abs=1e-15)
    assert np.all(ft > 0)
    assert np.allclose(ft, ft[::-1][np.r_[n_modes - 1, 0:n_modes - 1]], rtol=1e-14)  # even in k


def test_kernel_ft_bad_args(lib):
    with pytest.raises(nufft.DfsError):
        nufft.dfsnufft_kernel_ft(1, 2.3, 64, 32)


@pytest.mark.parametrize("w", [4, 6, 7, 8, 10, 13, 15])
def test_horner_kernel_fit(lib, w):
    """The per-tap polynomials the interpolation kernels evaluate match the kernel
    itself to within a few e^-beta (the kernel's own jump at its support edge)."""
    beta = 2.30 * w
    P = nufft.dfsnufft_es_horner(w, beta)
    assert P.shape == (w, w + 1)
    odd = w % 2
    c0 = (w - 1) // 2 if odd else w // 2 - 1
    mid = 0.0 if odd else 0.5
    ts = np.linspace(mid - 0.5, mid + 0.5 - 1e-12, 1001)
    worst = 0.0
    for a in range(w):
        acc = np.zeros_like(ts)
        for k in range(w, -1, -1):
            acc = acc * (ts - mid) + P[a, k]
        exact = np.array([nufft.dfsnufft_es_kernel((a - c0) - t, w, beta) for t in ts])
        worst = max(worst, float(np.max(np.abs(acc - exact))))
    assert worst < max(8 * math.exp(-beta), 2e-14), worst


def test_departure_and_rotation_argument_errors(lib):
    """Invalid sizes, iteration counts, dtypes, strides and null pointers are
    rejected before anything reaches a GPU (non-null dummies stand for device
    buffers; no kernel is launched)."""
    dummy = ctypes.c_void_p(16)
    bad_dep = [(7, 4, 1, 0, 3, 1e-4), (4, 4, 1, 0, 3, 1e-4), (8, 2, 1, 0, 3, 1e-4),
               (8, 4, 0, 0, 3, 1e-4), (8, 4, 1, 2, 3, 1e-4), (8, 4, 1, 0, 0, 1e-4),
               (8, 4, 1, 0, 65, 1e-4), (8, 4, 1, 0, 3, float("nan"))]
    for n_lon, n_lat, members, dtype, iters, dta in bad_dep:
        rc = lib.dfsnufft_departure_points(n_lon, n_lat, members, dtype, iters, dta, dummy,
                                           None, dummy, dummy, None, None)
        assert rc == nufft.ERR_INVALID_ARG, (n_lon, n_lat, members, dtype, iters, dta)
    assert lib.dfsnufft_departure_points(8, 4, 1, 0, 3, 1e-4, None, None, dummy, dummy,
                                         None, None) == nufft.ERR_INVALID_ARG
    rot = lib.dfsnufft_rotate_to_arrival
    assert rot(8, 4, 1, 0, dummy, dummy, None, dummy, dummy, 31, dummy, dummy,
               None) == nufft.ERR_INVALID_ARG                       # stride below n_lat n_lon
    assert rot(8, 4, 1, 0, dummy, None, None, dummy, dummy, 32, dummy, dummy,
               None) == nufft.ERR_INVALID_ARG                       # no points and no pq
    assert rot(9, 4, 1, 1, dummy, dummy, None, dummy, dummy, 36, dummy, dummy,
               None) == nufft.ERR_INVALID_ARG                       # odd n_lon
    assert rot(8, 4, 1, 1, None, None, dummy, None, dummy, 32, dummy, dummy,
               None) == nufft.ERR_INVALID_ARG                       # no u


def test_host_copy_bytes_argument_errors(lib):
    """A null plan or output pointer is rejected without touching a GPU."""
    out = [ctypes.c_int64() for _ in range(3)]
    refs = [ctypes.byref(o) for o in out]
    assert lib.dfsnufft_plan_host_copy_bytes(None, *refs) == nufft.ERR_INVALID_ARG
    dummy = ctypes.c_void_p(16)
    for k in range(3):
        args = list(refs)
        args[k] = None
        assert lib.dfsnufft_plan_host_copy_bytes(dummy, *args) == nufft.ERR_INVALID_ARG
