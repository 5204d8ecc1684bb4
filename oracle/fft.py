"""Oracle FFT: recursive mixed radix-2/3 Cooley-Tukey in float64.

Used for the Fourier-space Poisson solve of Eq. 2 and the force transform of
Eq. 3 (Sec. 2.1).  The paper's code calls FFTW3 / P3DFFT; the oracle writes
its own transform so that it shares nothing with the CUDA path.  Mesh edges
here are 2^a 3^b (tile edges such as 96 = 3 * 32), so a decimation-in-time
split by 2 or 3 suffices.

Definition (unnormalised, both directions):
    X[k] = sum_j x[j] exp(s 2 pi i j k / n),  s = -1 forward, +1 inverse.
Pinned against the O(n^2) DFT sum and numpy.fft (tests/test_oracle_fft.py).
"""
from __future__ import annotations

import numpy as np


def _fft_last(a: np.ndarray, sign: float) -> np.ndarray:
    n = a.shape[-1]
    if n == 1:
        return a.copy()
    if n % 2 == 0:
        p = 2
    elif n % 3 == 0:
        p = 3
    else:
        raise ValueError(f"length {n} is not of the form 2^a 3^b")
    # Decimation in time: sub-sequences a[p j + r], each transformed at length n/p,
    # recombined with twiddles exp(s 2 pi i r k / n) for k = 0..n-1.
    subs = [_fft_last(a[..., r::p], sign) for r in range(p)]
    k = np.arange(n)
    out = np.zeros(a.shape, dtype=np.complex128)
    for r in range(p):
        out += np.exp(sign * 2j * np.pi * r * k / n) * np.tile(subs[r], p)
    return out


def fft(a, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """Unnormalised DFT of ``a`` along ``axis`` (float64 complex)."""
    x = np.moveaxis(np.asarray(a, dtype=np.complex128), axis, -1)
    y = _fft_last(x, 1.0 if inverse else -1.0)
    return np.moveaxis(y, -1, axis)


def fft3(a, inverse: bool = False) -> np.ndarray:
    """Unnormalised 3-D DFT over the last three axes."""
    y = np.asarray(a, dtype=np.complex128)
    for ax in (-1, -2, -3):
        y = fft(y, axis=ax, inverse=inverse)
    return y


def dft_naive(a, inverse: bool = False) -> np.ndarray:
    """O(n^2) DFT along the last axis, straight from the definition."""
    x = np.asarray(a, dtype=np.complex128)
    n = x.shape[-1]
    j = np.arange(n)
    s = 1.0 if inverse else -1.0
    w = np.exp(s * 2j * np.pi * np.outer(j, j) / n)
    return x @ w.T
