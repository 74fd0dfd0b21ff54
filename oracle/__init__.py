"""Test oracle for the DFS spectral-interpolation step.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library path never does, and
it shares no code with the CUDA path.

Contents, each following the passage it cites:

* :func:`evaluate` -- the exact result the NUFFT approximates: plain FP64
  direct summation of Eq. 5.3 (type-II NUDFT, Sec. 5) in C (``dfs_oracle.c``),
  OpenMP over points, Neumaier-compensated sums.
* :func:`nudft_matrix` -- the same sum written as a dense NumPy matrix product,
  usable on tiny grids only (brute-force pin).
* :func:`complex_from_cossin` -- the map of Eq. 5.4 from the standard DFS
  cosine/sine coefficients (Eq. 4.6-4.7) to complex coefficients, with the
  rows the paper leaves out derived from the same expansion (n = 0 with a sine
  part, m = 0 with n >= 1).
* :func:`eval_cossin` -- direct evaluation of the standard DFS real form
  (Eq. 4.6-4.7), an independent route to the same field values.
* :func:`pr_to_std` -- the map from the partial-regularity DFS coefficients
  (Sec. 4, the expansion with sin(theta) and sin^2(theta) factors) to the
  standard DFS coefficients, in the paper's four cases (m = 0, m = 1, even
  m >= 2, odd m >= 3), with the one entry the product-to-sum identities fix
  differently from the printed list (f~_{0,m} = f_{1,m}/2 for even m >= 2).
* :func:`eval_pr` -- direct evaluation of the partial-regularity expansion
  (Sec. 4) from its own basis functions, the route that pins :func:`pr_to_std`.
* :func:`grid_to_coeffs` -- coefficients of Eq. 5.3 from samples on the Grid [0]
  arrival grid (Sec. 3): the samples extended to the doubled sphere by the
  field's parity (Sec. 4), then the plain discrete Fourier sums over the doubled
  torus (Sec. 4, the transforms in phi and theta written out as sums).

Submodules: :mod:`oracle.departure` (departure points of Eq. 2.4 and the
rotation Q of Sec. 2) and :mod:`oracle.lagrange` (the cubic and quintic
Lagrange interpolation of the paper's baseline, for the comparator).

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms, invariants and library special cases (see tests/test_oracle_pins.py,
tests/test_departure_pins.py and tests/test_lagrange_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdfsoracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (host code only, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.dfs_oracle_eval.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int]
        lib.dfs_oracle_eval.restype = ctypes.c_int
        lib.dfs_oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().dfs_oracle_max_threads())


def evaluate(coeffs: np.ndarray, lon: np.ndarray, colat: np.ndarray,
             nthreads: int = 0) -> np.ndarray:
    """Eq. 5.3 at every point, FP64.  ``coeffs`` is (N2, N1) or (F, N2, N1)
    complex in the centred layout (row n + N2/2, column m + N1/2).  Returns the
    complex values, shape (P,) or (F, P)."""
    lib = _load()
    c = np.ascontiguousarray(coeffs, dtype=np.complex128)
    single = c.ndim == 2
    if single:
        c = c[None]
    lon = np.ascontiguousarray(lon, dtype=np.float64)
    colat = np.ascontiguousarray(colat, dtype=np.float64)
    if lon.shape != colat.shape or lon.ndim != 1:
        raise ValueError("lon and colat must be 1-D of equal length")
    f, n2, n1 = c.shape
    out = np.empty((f, lon.size), dtype=np.complex128)
    for i in range(f):
        rc = lib.dfs_oracle_eval(n1, n2, c[i].ctypes.data, lon.size, lon.ctypes.data,
                                 colat.ctypes.data, out[i].ctypes.data, int(nthreads))
        if rc != 0:
            raise RuntimeError("dfs_oracle_eval failed with code %d" % rc)
    return out[0] if single else out


def nudft_matrix(coeffs: np.ndarray, lon: np.ndarray, colat: np.ndarray) -> np.ndarray:
    """Eq. 5.3 as a dense matrix-vector product (tiny grids only)."""
    c = np.asarray(coeffs, dtype=np.complex128)
    n2, n1 = c.shape
    n = np.arange(n2) - n2 // 2
    m = np.arange(n1) - n1 // 2
    a = np.exp(1j * (np.asarray(colat)[:, None, None] * n[None, :, None]
                     + np.asarray(lon)[:, None, None] * m[None, None, :]))
    return np.tensordot(a, c, axes=([1, 2], [0, 1]))


def complex_from_cossin(fc: np.ndarray, fs: np.ndarray, n_lon: int, n_lat: int) -> np.ndarray:
    """Eq. 5.4: standard DFS coefficients (index [n, m], n = 0..N, m = 0..M) to the
    centred complex array of shape (2 n_lat, n_lon).

    Even m multiply cos(n theta) (n >= 0), odd m multiply sin(n theta) (n >= 1),
    per Eq. 4.7.  Rows used exactly as printed: n >= 1 for every m >= 1 and
    n = 0, m = 0.  Rows derived from the same cos/sin expansion where the paper
    is silent or prints only part: f_{0,+-m} = (fc -+ i fs)/2 for even m >= 2,
    and f_{+-n,0} = fc_{n,0}/2 for n >= 1.
    """
    n2, n1 = 2 * n_lat, n_lon
    N, M = fc.shape[0] - 1, fc.shape[1] - 1
    if N >= n2 // 2 or M >= n1 // 2:
        raise ValueError("cos/sin truncation exceeds the complex array")
    out = np.zeros((n2, n1), dtype=np.complex128)
    r0, q0 = n2 // 2, n1 // 2

    def put(n, m, val):
        out[n + r0, m + q0] += val

    put(0, 0, fc[0, 0])
    for n in range(1, N + 1):
        put(n, 0, 0.5 * fc[n, 0])
        put(-n, 0, 0.5 * fc[n, 0])
    for m in range(1, M + 1):
        if m % 2 == 0:
            put(0, m, 0.5 * (fc[0, m] - 1j * fs[0, m]))
            put(0, -m, 0.5 * (fc[0, m] + 1j * fs[0, m]))
            for n in range(1, N + 1):
                for sn in (1, -1):
                    put(sn * n, m, 0.25 * (fc[n, m] - 1j * fs[n, m]))
                    put(sn * n, -m, 0.25 * (fc[n, m] + 1j * fs[n, m]))
        else:
            for n in range(1, N + 1):
                for sn in (1, -1):
                    put(sn * n, m, -sn * 0.25 * (1j * fc[n, m] + fs[n, m]))
                    put(sn * n, -m, -sn * 0.25 * (1j * fc[n, m] - fs[n, m]))
    return out


def eval_cossin(fc: np.ndarray, fs: np.ndarray, lon: np.ndarray, colat: np.ndarray) -> np.ndarray:
    """Eq. 4.6-4.7: f = sum_m [F^c_m(theta) cos m phi + F^s_m(theta) sin m phi] with
    F_m = sum_n f_{n,m} cos(n theta) for even m and sum_{n>=1} f_{n,m} sin(n theta)
    for odd m (the sine-in-phi part is absent for m = 0)."""
    lon = np.asarray(lon, dtype=np.float64)
    colat = np.asarray(colat, dtype=np.float64)
    N, M = fc.shape[0] - 1, fc.shape[1] - 1
    out = np.zeros(lon.shape, dtype=np.float64)
    for m in range(M + 1):
        if m % 2 == 0:
            basis = [np.cos(n * colat) for n in range(N + 1)]
            n_lo = 0
        else:
            basis = [np.sin(n * colat) for n in range(N + 1)]
            n_lo = 1
        fcm = sum(fc[n, m] * basis[n] for n in range(n_lo, N + 1))
        out += fcm * np.cos(m * lon)
        if m > 0:
            fsm = sum(fs[n, m] * basis[n] for n in range(n_lo, N + 1))
            out += fsm * np.sin(m * lon)
    return out


def pr_to_std(pc: np.ndarray, ps: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sec. 4: partial-regularity DFS coefficients f_{n,m} (index [n, m], n = 0..N,
    m = 0..M; cosine-in-phi part pc, sine part ps) to the standard DFS
    coefficients f~_{n,m} of Eq. 4.6-4.7 (same index range).

    Entries outside each case's range are ignored: m = 0 uses n = 0..N (cosine
    part only); m = 1 uses n = 0..N-1; even m >= 2 uses n = 1..N-1; odd m >= 3
    uses n = 1..N-2.  The four cases follow the paper; for even m >= 2 the
    printed f~_{0,m} = 0 is replaced by f_{1,m}/2, which the identity
    sin(t) sin(n t) = (cos((n-1)t) - cos((n+1)t))/2 gives at n = 1 (with 0 the
    expansion would not vanish at the poles, as its sin(theta) factor requires).
    """
    N, M = pc.shape[0] - 1, pc.shape[1] - 1
    if N < 6:
        raise ValueError("the case formulas of the paper need N >= 6")
    out = []
    for f in (pc, ps):
        g = np.zeros((N + 1, M + 1), dtype=np.float64)
        for m in range(M + 1):
            a = np.zeros(N + 3)                  # f_{n,m} on the case's range, zero elsewhere
            if m == 0:
                if f is ps:
                    continue
                g[:, 0] = f[:, 0]
                continue
            if m == 1:
                a[0:N] = f[0:N, 1]
                # sin t cos n t = (sin (n+1) t - sin (n-1) t) / 2
                g[1, 1] = 0.5 * (2.0 * a[0] - a[2])
                for n in range(2, N - 1):
                    g[n, 1] = 0.5 * (a[n - 1] - a[n + 1])
                for n in (N - 1, N):
                    g[n, 1] = 0.5 * a[n - 1]
            elif m % 2 == 0:
                a[1:N] = f[1:N, m]
                g[0, m] = 0.5 * a[1]
                g[1, m] = 0.5 * a[2]
                for n in range(2, N - 1):
                    g[n, m] = 0.5 * (-a[n - 1] + a[n + 1])
                for n in (N - 1, N):
                    g[n, m] = -0.5 * a[n - 1]
            else:
                a[1:N - 1] = f[1:N - 1, m]
                # sin^2 t sin n t = (2 sin n t - sin (n-2) t - sin (n+2) t) / 4
                g[1, m] = 0.25 * (3.0 * a[1] - a[3])
                g[2, m] = 0.25 * (2.0 * a[2] - a[4])
                for n in range(3, N - 2):
                    g[n, m] = 0.25 * (-a[n - 2] + 2.0 * a[n] - a[n + 2])
                for n in (N - 2, N - 1):
                    g[n, m] = 0.25 * (-a[n - 2] + 2.0 * a[n])
                g[N, m] = -0.25 * a[N - 2]
        out.append(g)
    return out[0], out[1]


def eval_pr(pc: np.ndarray, ps: np.ndarray, lon: np.ndarray, colat: np.ndarray) -> np.ndarray:
    """Sec. 4: f = sum_m F^c_m(theta) cos m phi + F^s_m(theta) sin m phi with
    F_0 = sum_{n=0}^N f_{n,0} cos n theta, F_1 = sum_{n=0}^{N-1} f_{n,1} sin theta cos n theta,
    F_m = sum_{n=1}^{N-1} f_{n,m} sin theta sin n theta (even m >= 2) and
    F_m = sum_{n=1}^{N-2} f_{n,m} sin^2 theta sin n theta (odd m >= 3)."""
    lon = np.asarray(lon, dtype=np.float64)
    colat = np.asarray(colat, dtype=np.float64)
    N, M = pc.shape[0] - 1, pc.shape[1] - 1
    st = np.sin(colat)
    out = np.zeros(lon.shape, dtype=np.float64)
    for m in range(M + 1):
        if m == 0:
            ns, basis = range(0, N + 1), lambda n: np.cos(n * colat)
        elif m == 1:
            ns, basis = range(0, N), lambda n: st * np.cos(n * colat)
        elif m % 2 == 0:
            ns, basis = range(1, N), lambda n: st * np.sin(n * colat)
        else:
            ns, basis = range(1, N - 1), lambda n: st * st * np.sin(n * colat)
        fcm = sum(pc[n, m] * basis(n) for n in ns)
        out += fcm * np.cos(m * lon)
        if m > 0:
            out += sum(ps[n, m] * basis(n) for n in ns) * np.sin(m * lon)
    return out


def grid_to_coeffs(samples: np.ndarray, parity) -> np.ndarray:
    """Sec. 3-4: samples f(phi_k, theta_j) of F fields on Grid [0] (shape (F, n_lat,
    n_lon); theta_j = (j + 1/2) pi / n_lat, phi_k = 2 pi k / n_lon) to the centred
    complex coefficients (F, 2 n_lat, n_lon) of the trigonometric interpolant on
    the doubled torus.

    Doubled sphere: rows j >= n_lat sit at theta_j in (pi, 2 pi), where the field
    is parity * f(phi + pi, 2 pi - theta), i.e. row 2 n_lat - 1 - j shifted by
    half a turn in longitude; parity is +1 for scalars and -1 for the wind
    components.  Then c_{n,m} = (1 / (N1 N2)) sum_{j,k} f_ext(phi_k, theta_j)
    exp(-i (m phi_k + n theta_j)), n = -N2/2..N2/2-1, m = -N1/2..N1/2-1."""
    samples = np.asarray(samples, dtype=np.float64)
    F, n_lat, n_lon = samples.shape
    n2, n1 = 2 * n_lat, n_lon
    parity = np.broadcast_to(np.asarray(parity, dtype=np.float64), (F,))
    th = (np.arange(n2) + 0.5) * (np.pi / n_lat)
    ph = np.arange(n1) * (2.0 * np.pi / n1)
    n = np.arange(n2) - n2 // 2
    m = np.arange(n1) - n1 // 2
    et = np.exp(-1j * np.outer(n, th))            # (modes n, rows j)
    ep = np.exp(-1j * np.outer(ph, m))            # (columns k, modes m)
    out = np.empty((F, n2, n1), dtype=np.complex128)
    for f in range(F):
        ext = np.empty((n2, n1))
        ext[:n_lat] = samples[f]
        for j in range(n_lat, n2):
            ext[j] = parity[f] * np.roll(samples[f][n2 - 1 - j], -(n1 // 2))
        out[f] = et @ ext @ ep / (n1 * n2)
    return out


def rel_linf(values: np.ndarray, reference: np.ndarray) -> float:
    """max |v - o| / max |o| over the checked points (the acceptance measure)."""
    v = np.asarray(values)
    o = np.asarray(reference)
    den = np.max(np.abs(o))
    return float(np.max(np.abs(v - o)) / (den if den > 0 else 1.0))
