"""Discrete Fourier transforms for the oracle (section 4.1).

Oracle -- test infrastructure only.
  dft_naive     -- the O(M^2) definition  X_l = sum_{k=0}^{M-1} exp(-2 pi i k l / M) x_k
                   (the printed upper limit N and the index label k are typos;
                   the sum runs over k = 0..M-1 for each l = 0..M-1).
  idft_naive    -- x_k = (1/M) sum_l exp(+2 pi i k l / M) X_l.
  fft_radix2    -- the oracle's own iterative radix-2 Cooley-Tukey FFT
                   (bit-reversal permutation, then log2 M butterfly stages),
                   forward or inverse (inverse includes the 1/M factor).
"""
from __future__ import annotations

import numpy as np


def dft_naive(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    M = x.size
    k = np.arange(M)
    kl = np.outer(k, k) % M  # reduce the exponent first so large M keeps full accuracy
    return np.exp(-2j * np.pi * kl / M) @ x


def idft_naive(X: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.complex128)
    M = X.size
    k = np.arange(M)
    kl = np.outer(k, k) % M
    return (np.exp(2j * np.pi * kl / M) @ X) / M


def _bit_reverse(M: int) -> np.ndarray:
    bits = M.bit_length() - 1
    idx = np.arange(M)
    rev = np.zeros(M, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_radix2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Radix-2 decimation-in-time FFT of a length-2^m vector."""
    x = np.asarray(x, dtype=np.complex128)
    M = x.size
    if M == 0 or M & (M - 1):
        raise ValueError("fft_radix2 needs a power-of-two length")
    a = x[_bit_reverse(M)].copy()
    sign = 1.0 if inverse else -1.0
    m = 2
    while m <= M:
        half = m // 2
        w = np.exp(sign * 2j * np.pi * np.arange(half) / m)
        blocks = a.reshape(M // m, m)
        even = blocks[:, :half].copy()
        odd = blocks[:, half:] * w
        blocks[:, :half] = even + odd
        blocks[:, half:] = even - odd
        m *= 2
    if inverse:
        a /= M
    return a


def ifft_radix2(X: np.ndarray) -> np.ndarray:
    return fft_radix2(X, inverse=True)
