"""Oracle power spectrum -- TEST INFRASTRUCTURE ONLY.

The compression test of Sec. 2.4 compares density and velocity power
spectra of two runs.  The spectrum of a real periodic field f on an n^3
mesh (box side n in mesh units) is taken as

    P(k) = < |F(k)|^2 > / n^6 * n^3,   F = the unnormalised DFT of f,

averaged over the modes whose |k| (in units of the fundamental 2 pi / n)
falls in each unit-width shell [j - 1/2, j + 1/2), j = 1 .. n/2, so that the
sum of P over all modes divided by n^3 is the variance of f (Parseval).  The
k = 0 mode is left out.  Pins: tests/test_oracle_power.py.
"""
from __future__ import annotations

import numpy as np


def mode_shells(n: int) -> np.ndarray:
    """Shell index round(|k|) of every mode of the full n^3 DFT ([z][y][x] order)."""
    m = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(m, m, m, indexing="ij")
    return np.rint(np.sqrt(kx * kx + ky * ky + kz * kz)).astype(np.int64)


def power_spectrum(field: np.ndarray):
    """(shell j = 1..n/2, P_j, modes per shell) of a real n^3 field."""
    f = np.asarray(field, np.float64)
    n = f.shape[0]
    F = np.fft.fftn(f)
    p = (np.abs(F) ** 2) / n ** 3
    shell = mode_shells(n)
    js = np.arange(1, n // 2 + 1)
    P = np.array([p[shell == j].mean() for j in js])
    cnt = np.array([(shell == j).sum() for j in js])
    return js, P, cnt
