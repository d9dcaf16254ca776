"""Heterogeneity index and heterogeneity matrix (section 6.4), by their definitions.

Oracle -- test infrastructure only.  0-based indices; f[0..N-1] is f_1..f_N.

g(F1, F2) (eq. g of section 6.4): with U_i, i in I, the left singular vectors
of the L-trajectory matrix of F1 and X_1..X_{K2} the L-lagged vectors of F2,
    g = sum_j dist^2(X_j, span U_I) / sum_j ||X_j||^2.
The distance is taken literally: the residual of the orthogonal projection
onto span U_I, whose squared norm is ||X_j||^2 - sum_i (U_i^T X_j)^2 for an
orthonormal U_I (the paper's second form).

H-matrix G_{B,T}: g_ij = g(base_i, test_j) with base_i = (f_i, ..., f_{i+B-1})
(i = 0..N-B) and test_j = (f_j, ..., f_{j+T-1}) (j = 0..N-T).  Reading: the
printed subseries F_{i,i+B} with F_{i,j} = (f_i..f_j) would hold B+1 samples
and run past f_N for the last i; the base and test lengths are B and T.

Index set I is 1-based as in the paper (I = {1, 2} are the two leading
triples).  A test window that is identically zero has g = 0 (the ratio is
0/0; nothing of it lies outside the subspace).
"""
from __future__ import annotations

import numpy as np

from . import jacobi, trajectory


def base_vectors(f1: np.ndarray, L: int, I) -> np.ndarray:
    """U_I: the left singular vectors i in I (1-based) of the L-trajectory matrix of f1."""
    X = trajectory.trajectory_matrix(np.asarray(f1, dtype=np.float64), L)
    U, s, Vt = jacobi.svd(X)
    order = np.argsort(-s, kind="stable")
    U = U[:, order]
    return U[:, [i - 1 for i in I]]


def heterogeneity(f1: np.ndarray, f2: np.ndarray, L: int, I) -> float:
    """g(F1, F2) by the distance definition."""
    U = base_vectors(f1, L, I)
    X2 = trajectory.trajectory_matrix(np.asarray(f2, dtype=np.float64), L)
    num = 0.0
    den = 0.0
    for j in range(X2.shape[1]):
        x = X2[:, j]
        r = x - U @ (U.T @ x)          # residual of the orthogonal projection
        num += float(r @ r)
        den += float(x @ x)
    return 0.0 if den == 0.0 else num / den


def hmatrix(f: np.ndarray, L: int, B: int, T: int, I) -> np.ndarray:
    """G_{B,T} with rows i = 0..N-B (base start) and columns j = 0..N-T (test start)."""
    f = np.asarray(f, dtype=np.float64)
    N = f.size
    if not (1 < L < B <= N and L <= T <= N):
        raise ValueError("need 1 < L < B <= N and L <= T <= N")
    if not I or min(I) < 1 or max(I) > min(L, B - L + 1) or len(set(I)) != len(I):
        raise ValueError("I must be distinct indices in 1..min(L, B-L+1)")
    G = np.empty((N - B + 1, N - T + 1))
    tests = [trajectory.trajectory_matrix(f[j:j + T], L) for j in range(N - T + 1)]
    for i in range(N - B + 1):
        U = base_vectors(f[i:i + B], L, I)
        for j, X2 in enumerate(tests):
            R = X2 - U @ (U.T @ X2)
            den = float(np.sum(X2 * X2))
            G[i, j] = 0.0 if den == 0.0 else float(np.sum(R * R)) / den
    return G
