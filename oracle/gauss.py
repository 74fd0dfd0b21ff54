"""Oracle for fields sampled on a Gauss-Legendre latitude grid (Sec. 3, the GL
grid; Sec. 5, interpolation for the spherical-harmonic model): the
coefficients of Eq. 5.3 from such samples, by the FFT in longitude and the
inversion of the DFT matrix in latitude.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library path never does, and
it shares no code with the CUDA path.  Plain FP64 NumPy.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre_colat(n_lat: int) -> np.ndarray:
    """Colatitudes theta_j = arccos(z_j) of the n_lat Gauss-Legendre nodes z_j
    (Sec. 3), in increasing order (from the north pole)."""
    z, _ = np.polynomial.legendre.leggauss(n_lat)
    return np.sort(np.arccos(z))


def doubled_colat(colat: np.ndarray) -> np.ndarray:
    """The 2 n_lat rows of the doubled circle: theta_j, then the mirrored rows
    -theta_{2 n_lat - 1 - j} (the same order as the Grid [0] extension)."""
    colat = np.asarray(colat, dtype=np.float64)
    return np.concatenate([colat, -colat[::-1]])


def gl_to_coeffs(samples: np.ndarray, parity, colat: np.ndarray) -> np.ndarray:
    """Samples (F, n_lat, n_lon) at the colatitudes ``colat`` (n_lat values in
    (0, pi)) and phi_k = 2 pi k / n_lon to the centred coefficients (F, 2 n_lat,
    n_lon) of Eq. 5.3.  The samples are extended to the doubled sphere by the
    field's parity (Sec. 4: row 2 n_lat - 1 - j is the point (phi + pi, -theta_j),
    value parity * f); then for every longitude mode m (the FFT of the rows,
    divided by n_lon) the 2 n_lat latitude coefficients solve V c = g with the
    DFT matrix V_{j,n} = exp(i n theta_j) of the doubled rows, n = -n_lat..n_lat-1."""
    samples = np.asarray(samples, dtype=np.float64)
    F, n_lat, n_lon = samples.shape
    n2, n1 = 2 * n_lat, n_lon
    parity = np.broadcast_to(np.asarray(parity, dtype=np.float64), (F,))
    th = doubled_colat(colat)
    n = np.arange(n2) - n2 // 2
    V = np.exp(1j * np.outer(th, n))                 # (rows j, modes n)
    out = np.empty((F, n2, n1), dtype=np.complex128)
    for f in range(F):
        ext = np.empty((n2, n1))
        ext[:n_lat] = samples[f]
        for j in range(n_lat, n2):
            ext[j] = parity[f] * np.roll(samples[f][n2 - 1 - j], -(n1 // 2))
        g = np.fft.fftshift(np.fft.fft(ext, axis=1), axes=1) / n1    # (rows, modes m)
        out[f] = np.linalg.solve(V, g)
    return out
