"""Algorithms 2, 3 and 4 of the paper on the oracle's own radix-2 FFT.

Oracle -- test infrastructure only.  0-based indices; f[0..N-1] is f_1..f_N.

Readings of the printed text (each is pinned by a test against the explicit
trajectory matrix):
  * Algorithm 2, step 1 defines c = (f_{N-L+1}, ..., f_N, f_1, ..., f_{N-L});
    the case formula printed just before it has an off-by-one in its second
    case, so the algorithm's step is followed.
  * FFT length: the paper uses exactly N.  Any M >= N gives the same products
    when M - N zeros are placed between the two blocks of c (the circulant
    then embeds the same Toeplitz matrix).  The oracle uses the next power of
    two >= 2N so that it never shares the CUDA path's choice of M.
  * Algorithm 3 prints the output slice p'_{L-1}..p'_N (K+1 entries); the
    correct slice is p'_L..p'_N (1-based), i.e. indices M-K..M-1 here.
  * Algorithm 4 prints g = sigma (w . g'); comparing with the convolution
    identity of section 5 (g_k = c_k (u'*v')_k with c_k the reciprocal
    antidiagonal counts), the counts must divide, not multiply.
"""
from __future__ import annotations

import numpy as np

from .dft import fft_radix2, ifft_radix2
from .trajectory import antidiagonal_counts


def _ffts(fft: str):
    """(forward, inverse) complex FFTs with the definitions of section 4.1 (inverse with 1/M).

    "radix2" is the oracle's own FFT; "library" is numpy's, for sizes where the
    pure-Python butterfly stages are too slow (pinned to "radix2" by a test).
    """
    if fft == "radix2":
        return fft_radix2, ifft_radix2
    if fft == "library":
        return np.fft.fft, np.fft.ifft
    raise ValueError(f"unknown fft {fft!r}")


def fft_length(N: int) -> int:
    """Oracle FFT length: the next power of two >= 2N."""
    M = 1
    while M < 2 * N:
        M *= 2
    return M


def circulant_column(f: np.ndarray, L: int, M: int) -> np.ndarray:
    """First column c of the circulant embedding (Algorithm 2 step 1, zero-padded to M)."""
    f = np.asarray(f, dtype=np.float64)
    N = f.size
    if M < N:
        raise ValueError("M must be >= N")
    c = np.zeros(M)
    c[:L] = f[N - L:]            # f_{N-L+1}..f_N
    c[L + (M - N):] = f[:N - L]  # f_1..f_{N-L}, after the M-N inserted zeros
    return c


def spectrum(f: np.ndarray, L: int, M: int, fft: str = "radix2") -> np.ndarray:
    """c-hat = FFT_M(c) (Algorithm 2 step 2), computed once per (f, L)."""
    fwd, _ = _ffts(fft)
    return fwd(circulant_column(f, L, M))


def hankel_matvec(chat: np.ndarray, N: int, L: int, v: np.ndarray, fft: str = "radix2") -> np.ndarray:
    """Algorithm 2: p = X v for v of length K."""
    fwd, inv = _ffts(fft)
    M = chat.size
    K = N - L + 1
    w = np.zeros(M)
    w[:K] = np.asarray(v, dtype=np.float64)[::-1]     # (v_K, ..., v_1, 0, ..., 0)
    p = inv(fwd(w) * chat)
    return p[:L].real                                  # p'_1..p'_L


def hankel_rmatvec(chat: np.ndarray, N: int, L: int, u: np.ndarray, fft: str = "radix2") -> np.ndarray:
    """Algorithm 3: p = X^T u for u of length L."""
    fwd, inv = _ffts(fft)
    M = chat.size
    K = N - L + 1
    w = np.zeros(M)
    w[M - L:] = np.asarray(u, dtype=np.float64)[::-1]  # (0, ..., 0, u_L, ..., u_1)
    p = inv(fwd(w) * chat)
    return p[M - K:].real                              # p'_L..p'_N when M = N


def rank1_hankelization(sigma: float, u: np.ndarray, v: np.ndarray, M: int | None = None,
                        fft: str = "radix2") -> np.ndarray:
    """Algorithm 4: diagonal average of sigma u v^T via a linear convolution."""
    fwd, inv = _ffts(fft)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    L, K = u.size, v.size
    N = L + K - 1
    if M is None:
        M = fft_length(N)
    if M < N:
        raise ValueError("M must be >= L + K - 1 for a linear convolution")
    up = np.zeros(M)
    up[:L] = u
    vp = np.zeros(M)
    vp[:K] = v
    g = inv(fwd(vp) * fwd(up)).real[:N]
    return sigma * g / antidiagonal_counts(N, L)
