"""Seeded synthetic series shaped like the paper's workloads.

This module holds the input generators only: it draws series, lengths,
windows and arrival times.  It contains none of the SSA arithmetic (no
embedding, no FFT, no SVD, no Hankelization), so both the CUDA path and the
CPU oracle can consume its output without sharing any of the method.

Randomness comes from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: value i
of stream s under seed S is mix(S_s + (i+1)*GAMMA), where S_s is the s-th
output of a splitmix64 sequence seeded with S.  Uniforms take the top 53
bits; normals use the Box-Muller transform.

Workloads (sizes follow the paper's experiments, section 6 and 7):
  * ``three_sines``   N=1000-style series: three sinusoids (periods 12, 37.5
    and 101; amplitudes 2, 1, 0.5; random phases) + exponential trend +
    N(0, 0.1^2) noise.
  * ``many_sines``    long series: 20 sinusoids with periods log-uniform in
    [5, 5000] and amplitudes 1/i, trend and N(0, 0.1^2) noise.
  * ``damped_sines``  exact-rank-40 sum of 20 damped cosines plus tiny noise.
  * ``geometric`` / ``cosine``: closed-form series used as pins.
  * ``bootstrap_series`` / ``hmatrix_series``: the series of section 6.3/6.4.
The exponential trend 0.01*1.001^n overflows double precision near
n = 7e5, so for N != 1000 it is evaluated as 0.01*1.001^(1000 n / N), which
keeps the N = 1000 shape at every length.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of stream ``stream``: the (stream+1)-th splitmix64 output for ``seed``."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + GAMMA * np.uint64(stream + 1)
    return _mix(np.array([s], dtype=np.uint64))[0]


def raw64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    key = stream_key(seed, stream)
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + GAMMA * i)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits."""
    return (raw64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller from two uniform streams."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 1, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def trend(n: np.ndarray, N: int) -> np.ndarray:
    if N == 1000:
        return 0.01 * 1.001 ** n
    return 0.01 * 1.001 ** (1000.0 * n / N)


def three_sines(N: int, seed: int = 0, noise: float = 0.1) -> np.ndarray:
    n = np.arange(1, N + 1, dtype=np.float64)
    ph = 2.0 * math.pi * uniform(seed, 0, 3)
    f = (2.0 * np.sin(2 * math.pi * n / 12.0 + ph[0])
         + 1.0 * np.sin(2 * math.pi * n / 37.5 + ph[1])
         + 0.5 * np.sin(2 * math.pi * n / 101.0 + ph[2])
         + trend(n, N))
    if noise:
        f = f + noise * normal(seed, 10, N)
    return f


def many_sines(N: int, seed: int = 1, n_periods: int = 20, noise: float = 0.1) -> np.ndarray:
    n = np.arange(1, N + 1, dtype=np.float64)
    lp = math.log(5.0) + (math.log(5000.0) - math.log(5.0)) * uniform(seed, 0, n_periods)
    periods = np.exp(lp)
    ph = 2.0 * math.pi * uniform(seed, 1, n_periods)
    f = trend(n, N).copy()
    for i in range(n_periods):
        f += (1.0 / (i + 1)) * np.sin(2 * math.pi * n / periods[i] + ph[i])
    if noise:
        f = f + noise * normal(seed, 10, N)
    return f


def damped_sines(N: int, seed: int = 3, n_pairs: int = 20, noise: float = 1e-6) -> np.ndarray:
    n = np.arange(1, N + 1, dtype=np.float64)
    rho = 0.9999 + 0.0001 * uniform(seed, 0, n_pairs)
    lp = math.log(5.0) + (math.log(5000.0) - math.log(5.0)) * uniform(seed, 1, n_pairs)
    omega = 2 * math.pi / np.exp(lp)
    ph = 2.0 * math.pi * uniform(seed, 2, n_pairs)
    f = np.zeros(N)
    for i in range(n_pairs):
        f += np.exp(n * math.log(rho[i])) * np.cos(omega[i] * n + ph[i])
    if noise:
        f = f + noise * normal(seed, 10, N)
    return f


def geometric(N: int, a: float) -> np.ndarray:
    """f_n = a^n, n = 1..N (a rank-1 series)."""
    return a ** np.arange(1, N + 1, dtype=np.float64)


def cosine(N: int, T: int, A: float = 1.0, phi: float = 0.3) -> np.ndarray:
    """f_n = A cos(2 pi n / T + phi), n = 1..N (a rank-2 series for T > 2)."""
    n = np.arange(1, N + 1, dtype=np.float64)
    return A * np.cos(2 * math.pi * n / T + phi)


def bootstrap_series(N: int, seed: int, sigma: float = 5.0) -> np.ndarray:
    """Section 6.3 series (rank 5) plus N(0, sigma^2) noise.

    The paper's middle terms read sin(2 pi/13 * n/N); that has period 13N and
    contradicts the stated rank 5, so periods 13 and 37 in n are used.
    """
    n = np.arange(1, N + 1, dtype=np.float64)
    f = 10 * np.exp(-5 * n / N) + np.sin(2 * math.pi * n / 13) + 2.5 * np.sin(2 * math.pi * n / 37)
    return f + sigma * normal(seed, 10, N)


def hmatrix_series(N: int, Q: int, seed: int = 0) -> np.ndarray:
    """Section 6.4 series: a sinusoid whose period changes from 10 to 10.5 at n = Q."""
    n = np.arange(1, N + 1, dtype=np.float64)
    f = np.where(n < Q, np.sin(2 * math.pi * n / 10), np.sin(2 * math.pi * n / 10.5))
    return f + 0.01 * normal(seed, 10, N)


def batch_workload(count: int = 4096, seed: int = 2, n_lo: int = 500, n_hi: int = 20000,
                   k_lo: int = 4, k_hi: int = 32):
    """Ragged batch: N ~ U{n_lo..n_hi}, L alternating round(N/3) and N//2, k ~ U{k_lo..k_hi}.

    Returns (series list, L array, k array); series i uses the three-sine
    generator with seed ``seed*1_000_003 + i``.
    """
    u = uniform(seed, 0, count)
    Ns = (n_lo + np.floor(u * (n_hi - n_lo + 1))).astype(np.int64)
    Ls = np.where(np.arange(count) % 2 == 0, np.floor(Ns / 3 + 0.5), Ns // 2).astype(np.int64)
    uk = uniform(seed, 1, count)
    ks = (k_lo + np.floor(uk * (k_hi - k_lo + 1))).astype(np.int64)
    series = [three_sines(int(Ns[i]), seed=seed * 1_000_003 + i) for i in range(count)]
    return series, Ls, ks


def serving_arrivals(rate: float, duration: float, seed: int = 4, n_lo: float = 1e3,
                     n_hi: float = 1e6, k_lo: int = 2, k_hi: int = 64):
    """Poisson arrivals: (t_arrival, N, L, k, seed) tuples, N log-uniform, L = N//2."""
    count = int(rate * duration * 1.5) + 16
    gaps = -np.log1p(-uniform(seed, 0, count)) / rate
    t = np.cumsum(gaps)
    t = t[t < duration]
    m = len(t)
    Ns = np.floor(np.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * uniform(seed, 1, m))).astype(np.int64)
    ks = (k_lo + np.floor(uniform(seed, 2, m) * (k_hi - k_lo + 1))).astype(np.int64)
    return [(float(t[i]), int(Ns[i]), int(Ns[i] // 2), int(ks[i]), int(seed * 10_000_019 + i)) for i in range(m)]
