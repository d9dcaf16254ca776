"""Explicit trajectory matrix, explicit products and naive diagonal averaging.

Oracle -- test infrastructure only.  Indices are 0-based here: the paper's
f_1..f_N is f[0..N-1].
  trajectory_matrix  -- section 2.1: the L x K Hankel matrix, X[i, j] = f[i+j].
  matvec / rmatvec   -- X v and X^T u by forming X (the O(LK) product the fast
                        method replaces, section 4).
  antidiagonal_counts-- number of entries on each antidiagonal (the constants
                        of the three cases in section 2.4): min(n+1, L, K, N-n).
  diagonal_average   -- section 2.4, the three-case formula written out, for
                        any L x K matrix Y (L > K handled by transposing, since
                        antidiagonals of Y and Y^T coincide).
"""
from __future__ import annotations

import numpy as np


def trajectory_matrix(f: np.ndarray, L: int) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    N = f.size
    K = N - L + 1
    i = np.arange(L)[:, None]
    j = np.arange(K)[None, :]
    return f[i + j]


def matvec(f: np.ndarray, L: int, v: np.ndarray) -> np.ndarray:
    return trajectory_matrix(f, L) @ np.asarray(v, dtype=np.float64)


def rmatvec(f: np.ndarray, L: int, u: np.ndarray) -> np.ndarray:
    return trajectory_matrix(f, L).T @ np.asarray(u, dtype=np.float64)


def antidiagonal_counts(N: int, L: int) -> np.ndarray:
    K = N - L + 1
    n = np.arange(N)
    return np.minimum(np.minimum(n + 1, N - n), min(L, K)).astype(np.float64)


def diagonal_average(Y: np.ndarray) -> np.ndarray:
    """g_k of section 2.4 for an L x K matrix Y (1-based k in the comments)."""
    Y = np.asarray(Y, dtype=np.float64)
    L, K = Y.shape
    if L > K:
        return diagonal_average(Y.T)
    N = L + K - 1
    g = np.empty(N)
    for k1 in range(1, N + 1):          # paper's k = 1..N
        if k1 <= L:                     # 1 <= k <= L: j = 1..k, divide by k
            j1 = np.arange(1, k1 + 1)
            denom = k1
        elif k1 < K:                    # L < k < K: j = 1..L, divide by L
            j1 = np.arange(1, L + 1)
            denom = L
        else:                           # K <= k <= N: j = k-K+1..L, divide by N-k+1
            j1 = np.arange(k1 - K + 1, L + 1)
            denom = N - k1 + 1
        # y_{j, k-j+1} (1-based) is Y[j-1, k-j] (0-based)
        g[k1 - 1] = Y[j1 - 1, k1 - j1].sum() / denom
    return g
