"""Oracle FFT (own radix-2 / direct DFT) pinned against numpy.fft."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 3, 6, 24])
def test_fft1d_matches_numpy(oracle, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(oracle.fft1d(x, -1), np.fft.fft(x), rtol=0, atol=1e-13 * n)
    np.testing.assert_allclose(oracle.fft1d(x, +1), n * np.fft.ifft(x), rtol=0, atol=1e-13 * n)


@pytest.mark.parametrize("n", [4, 8, 16, 24])
def test_fft3d_matches_numpy_and_round_trips(oracle, n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    X = oracle.fft3d(x, -1)
    np.testing.assert_allclose(X, np.fft.fftn(x), rtol=0, atol=1e-12 * n ** 3)
    back = oracle.fft3d(X, +1) / n ** 3
    np.testing.assert_allclose(back, x, rtol=0, atol=1e-13)
