"""Pins for the oracle's DFT/FFT (section 4.1) against facts fixed by the mathematics."""
import numpy as np
import pytest

from oracle import dft


def test_dft_hand_example(golden):
    g = golden("dft_length4.txt")
    X = dft.dft_naive(g["x"])
    np.testing.assert_allclose(X.real, g["X_re"], atol=1e-13)
    np.testing.assert_allclose(X.imag, g["X_im"], atol=1e-13)
    Xf = dft.fft_radix2(g["x"])
    np.testing.assert_allclose(Xf.real, g["X_re"], atol=1e-13)
    np.testing.assert_allclose(Xf.imag, g["X_im"], atol=1e-13)


@pytest.mark.parametrize("M", [1, 2, 4, 8, 16, 64, 256, 1024])
def test_radix2_matches_naive_dft(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    ref = dft.dft_naive(x)
    got = dft.fft_radix2(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    back = dft.ifft_radix2(got)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))
    np.testing.assert_allclose(dft.idft_naive(ref), x, atol=1e-12)


@pytest.mark.parametrize("M", [2 ** 12, 2 ** 16])
def test_radix2_matches_library_fft(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    ref = np.fft.fft(x)
    got = dft.fft_radix2(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_parseval_delta_and_hermitian():
    M = 512
    rng = np.random.default_rng(1)
    x = rng.standard_normal(M)
    X = dft.fft_radix2(x)
    # Parseval: sum |x|^2 = (1/M) sum |X|^2
    assert abs(np.sum(x * x) - np.sum(np.abs(X) ** 2) / M) <= 1e-12 * np.sum(x * x)
    # real input -> Hermitian output X_{M-l} = conj(X_l)
    assert np.max(np.abs(X[1:][::-1] - np.conj(X[1:]))) <= 1e-12 * np.max(np.abs(X))
    # delta -> constant, constant -> M * delta
    e = np.zeros(M)
    e[0] = 1.0
    np.testing.assert_allclose(dft.fft_radix2(e), np.ones(M), atol=1e-15)
    c = dft.fft_radix2(np.ones(M))
    assert abs(c[0] - M) < 1e-10 and np.max(np.abs(c[1:])) < 1e-10
    # shift theorem: x shifted by s multiplies X by exp(-2 pi i l s / M)
    s = 37
    Xs = dft.fft_radix2(np.roll(x, s))
    l = np.arange(M)
    np.testing.assert_allclose(Xs, X * np.exp(-2j * np.pi * l * s / M), atol=1e-11)


def test_non_power_of_two_rejected():
    with pytest.raises(ValueError):
        dft.fft_radix2(np.ones(12))
