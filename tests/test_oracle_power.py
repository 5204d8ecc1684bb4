"""Pins for the oracle power spectrum: a single plane wave puts all its power
in the shell of its wavenumber with the closed-form amplitude, and Parseval
ties the total over modes to the variance of the field."""
import numpy as np

from oracle import power


def test_plane_wave_power_in_one_shell():
    n, A, k = 16, 0.7, 3
    x = np.arange(n)
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    f = A * np.cos(2 * np.pi * k * xx / n)
    js, P, cnt = power.power_spectrum(f)
    # F(+-k) = A n^3 / 2 on two modes of shell 3: p = (A n^3 / 2)^2 / n^3 each
    expect = 2 * (A * n ** 3 / 2) ** 2 / n ** 3 / cnt[k - 1]
    np.testing.assert_allclose(P[k - 1], expect, rtol=1e-12)
    assert np.all(P[np.arange(len(P)) != k - 1] < 1e-20)


def test_parseval():
    rng = np.random.default_rng(5)
    n = 12
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    F = np.fft.fftn(f)
    total = np.sum(np.abs(F) ** 2) / n ** 3
    np.testing.assert_allclose(total / n ** 3, f.var(), rtol=1e-12)
    js, P, cnt = power.power_spectrum(f)
    shell = power.mode_shells(n)
    inside = np.sum(cnt * P)
    outside = np.sum((np.abs(F) ** 2 / n ** 3)[(shell > n // 2) | (shell == 0)])
    np.testing.assert_allclose(inside + outside, total, rtol=1e-12)
