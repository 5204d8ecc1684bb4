"""Oracle Poisson solves: Eqs. 1-3 and the two-level split of Sec. 2.1.

Eq. 1: lap(phi) = 4 pi G rho.  Eq. 2: phi(k) = -4 pi G rho(k) / k^2.
Eq. 3: F(k) = -i m phi(k) k; three inverse transforms give the force.
So the acceleration a = F/m has a(k) = 4 pi G i k rho(k) / k^2.

Sec. 2.1 splits this into a long-range term on a coarse mesh (n_g = n_p/2
cells per side) and a short-range term on a mesh four times finer that is
local to each tile (with a buffer, Fig. 1).  The paper defers the split's
kernels to earlier work, so the oracle takes the Gaussian split:

  long range  (coarse mesh):  a(k) = 4 pi G i k exp(-k^2 r_s^2) rho(k) / k^2
  short range (fine tiles):   K(r) = -G r S(r) / r^3 for 0 < r <= R, else 0,
                              S(r) = erfc(r / 2 r_s) + r/(r_s sqrt(pi)) exp(-r^2 / 4 r_s^2),
  which sum to the Newtonian force for r <= R (up to S(R) and mesh effects).

Units: lengths in fine cells, masses as deposited.  On a periodic mesh of n
points with spacing h fine cells, a mass M(j) per cell has the density
Fourier coefficient rho_m = DFT[M](m) / V with V = (n h)^3 and k = 2 pi m /
(n h).  Readings where the paper is silent: k = 0 is dropped (mean density
removed); at the Nyquist index the gradient factor k_d is set to 0 (k^2
keeps its full value) so the force stays real; no CIC deconvolution.

Pins: tests/test_oracle_solve.py (plane waves, brute-force real-space
convolution for the tile kernel, momentum conservation, 1/r^2; the one-mode
forms against the definition, the full transform and a plane wave).
"""
from __future__ import annotations

import math

import numpy as np

from .fft import fft3


def mode_numbers(n: int) -> np.ndarray:
    """Signed DFT mode numbers 0..n/2, -(n/2-1)..-1 (n/2 kept positive)."""
    j = np.arange(n)
    return np.where(j <= n // 2, j, j - n)


def accel_periodic(M: np.ndarray, h: float, G: float, r_s: float = 0.0) -> np.ndarray:
    """Acceleration [3, n, n, n] at the points of a periodic mesh of spacing h
    carrying masses M [n, n, n] (indexed [z, y, x]); r_s > 0 keeps only the
    Gaussian long-range part."""
    n = M.shape[0]
    V = (n * h) ** 3
    m = mode_numbers(n)
    k1 = 2.0 * np.pi * m / (n * h)
    kgrad = np.where(np.abs(m) == n // 2, 0.0, k1) if n % 2 == 0 else k1
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    g = np.zeros_like(k2)
    nz = k2 > 0
    g[nz] = 4.0 * np.pi * G / (k2[nz] * V)
    if r_s > 0:
        g *= np.exp(-k2 * r_s * r_s)
    Mk = fft3(M)
    gz, gy, gx = np.meshgrid(kgrad, kgrad, kgrad, indexing="ij")
    out = np.empty((3, n, n, n))
    for d, kd in enumerate((gx, gy, gz)):
        out[d] = fft3(1j * kd * g * Mk, inverse=True).real
    return out


def dft_mode(F: np.ndarray, m) -> complex:
    """One coefficient of the unnormalised forward 3-D DFT of a real field F
    [n, n, n] ([z, y, x]) at mode numbers m = (mx, my, mz), straight from the
    definition sum_c F(c) exp(-2 pi i m.c / n), summed one axis at a time."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    j = np.arange(n)
    ex, ey, ez = (np.exp(-2j * np.pi * mm * j / n) for mm in m)
    t = F @ ex.real + 1j * (F @ ex.imag)          # [z, y]
    return complex(ez @ (t @ ey))


def accel_mode(M: np.ndarray, h: float, G: float, r_s: float, m) -> np.ndarray:
    """The DFT coefficient at mode numbers m = (mx, my, mz) of the three
    components of accel_periodic(M, h, G, r_s), from Eqs. 2-3 at that one wave
    vector: n^3 i k_d g(k) DFT[M](m), g = 4 pi G exp(-k^2 r_s^2) / (k^2 V),
    with the same readings (0 at k = 0, k_d = 0 at the Nyquist index).  For
    meshes too large for a full oracle transform."""
    n = M.shape[0]
    V = (n * h) ** 3
    mm = [((int(c) + n // 2) % n) - n // 2 if (int(c) % n) != n // 2 else n // 2 for c in m]
    k = np.array([2.0 * np.pi * c / (n * h) for c in mm])
    kgrad = np.array([0.0 if 2 * abs(c) == n else kd for c, kd in zip(mm, k)])
    k2 = float(np.sum(k * k))
    if k2 == 0.0:
        return np.zeros(3, dtype=np.complex128)
    g = 4.0 * np.pi * G / (k2 * V)
    if r_s > 0:
        g *= math.exp(-k2 * r_s * r_s)
    return n ** 3 * 1j * kgrad * g * dft_mode(M, m)


def short_range_shape(r: np.ndarray, r_s: float) -> np.ndarray:
    """S(r) of the Gaussian split: the fraction of the Newtonian force kept at short range."""
    erfc = np.vectorize(math.erfc)
    return erfc(r / (2.0 * r_s)) + r / (r_s * math.sqrt(math.pi)) * np.exp(-r * r / (4.0 * r_s * r_s))


def fine_kernel(T: int, G: float, r_s: float, R: float) -> np.ndarray:
    """Real-space short-range vector kernel [3, T, T, T] on a tile, minimal-image
    separations; acceleration at c from unit mass at c' is K(c - c')."""
    m = mode_numbers(T).astype(np.float64)   # separations -(T/2-1)..T/2
    rz, ry, rx = np.meshgrid(m, m, m, indexing="ij")
    r = np.sqrt(rx * rx + ry * ry + rz * rz)
    K = np.zeros((3, T, T, T))
    sel = (r > 0) & (r <= R)
    coef = np.zeros_like(r)
    coef[sel] = -G * short_range_shape(r[sel], r_s) / r[sel] ** 3
    for d, rd in enumerate((rx, ry, rz)):
        K[d] = coef * rd
    return K


def accel_tile(rho_tile: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Circular convolution a_d = K_d * rho on a T^3 tile via the oracle FFT."""
    T = rho_tile.shape[0]
    rk = fft3(rho_tile)
    out = np.empty((3, T, T, T))
    for d in range(3):
        out[d] = fft3(fft3(K[d]) * rk, inverse=True).real / T ** 3
    return out
