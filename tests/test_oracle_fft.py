"""Pins for the oracle FFT (Sec. 2.1 Fourier transforms): the O(n^2) DFT
definition, numpy's FFT as an independent library routine, Parseval and the
inverse relation."""
import numpy as np
import pytest

from oracle import fft as offt


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27, 32, 48])
@pytest.mark.parametrize("inverse", [False, True])
def test_matches_naive_dft(n, inverse):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((5, n)) + 1j * rng.standard_normal((5, n))
    np.testing.assert_allclose(offt.fft(x, inverse=inverse), offt.dft_naive(x, inverse=inverse),
                               rtol=0, atol=1e-11 * n)


@pytest.mark.parametrize("n", [64, 96, 128, 192, 384])
def test_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    np.testing.assert_allclose(offt.fft(x), np.fft.fft(x), rtol=0, atol=1e-10 * n)
    np.testing.assert_allclose(offt.fft(x, inverse=True), np.fft.ifft(x) * n, rtol=0, atol=1e-10 * n)


def test_parseval_and_inverse():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((4, 96)) + 1j * rng.standard_normal((4, 96))
    X = offt.fft(x)
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2, axis=1), 96 * np.sum(np.abs(x) ** 2, axis=1), rtol=1e-12)
    np.testing.assert_allclose(offt.fft(X, inverse=True) / 96, x, atol=1e-12)


def test_fft3_matches_numpy_fftn():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((12, 8, 6))
    np.testing.assert_allclose(offt.fft3(x), np.fft.fftn(x), atol=1e-10)


def test_single_mode_closed_form():
    n = 96
    j = np.arange(n)
    m = 5
    X = offt.fft(np.exp(2j * np.pi * m * j / n))
    expect = np.zeros(n, complex)
    expect[m] = n
    np.testing.assert_allclose(X, expect, atol=1e-10)


def test_rejects_bad_length():
    with pytest.raises(ValueError):
        offt.fft(np.ones(10 * 7))
