"""Pins of the oracle's heterogeneity index and H-matrix (section 6.4)."""
import math

import numpy as np
import pytest

from oracle import hmatrix, trajectory


def _sine(n, period):
    return np.sin(2 * math.pi * np.arange(1, n + 1) / period)


def test_range_and_exact_zero_for_the_same_structure():
    # a noise-free sinusoid: its lagged vectors span exactly the two leading vectors
    f1 = _sine(60, 10)
    f2 = _sine(45, 10)[7:]                      # same frequency, other phase and length
    assert abs(hmatrix.heterogeneity(f1, f2, 20, [1, 2])) <= 1e-12
    g = hmatrix.heterogeneity(f1, _sine(45, 10.5), 20, [1, 2])
    assert 1e-4 < g < 1.0


def test_full_subspace_gives_zero():
    rng = np.random.default_rng(1)
    f1 = rng.standard_normal(40)                # K1 = 31 >= L: the L-trajectory matrix has rank L
    f2 = rng.standard_normal(30)
    L = 10
    assert abs(hmatrix.heterogeneity(f1, f2, L, list(range(1, L + 1)))) <= 1e-12


def test_orthogonal_structure_gives_one():
    # period-4 cosine: lagged vectors span {(1,0,-1,0), (0,1,0,-1)} in R^4;
    # (-1)^n has lagged vectors +-(1,-1,1,-1), orthogonal to that span
    n = np.arange(1, 41)
    f1 = np.cos(2 * math.pi * n / 4)
    f2 = (-1.0) ** n[:12]
    assert abs(hmatrix.heterogeneity(f1, f2, 4, [1, 2]) - 1.0) <= 1e-12


def test_matches_lapack_projection():
    rng = np.random.default_rng(3)
    f = np.cumsum(rng.standard_normal(90)) * 0.1 + _sine(90, 7)
    L, B, T, I = 12, 30, 25, [1, 3]
    G = hmatrix.hmatrix(f, L, B, T, I)
    assert G.shape == (90 - B + 1, 90 - T + 1)
    for i, j in [(0, 0), (5, 40), (60, 65), (33, 12)]:
        U, s, _ = np.linalg.svd(trajectory.trajectory_matrix(f[i:i + B], L), full_matrices=False)
        Ui = U[:, [0, 2]]
        X = trajectory.trajectory_matrix(f[j:j + T], L)
        num = np.sum(X * X) - np.sum((Ui.T @ X) ** 2)
        assert abs(G[i, j] - num / np.sum(X * X)) <= 1e-12


def test_step_change_zero_pattern():
    """Noise-free version of the section 6.4 series: g_ij = 0 exactly when the
    base and the test window lie on the same side of the change at n = Q, and
    > 0 when they lie on different sides.  A window of the wrong length or
    start shifts this pattern."""
    N, Q, B, T, L = 80, 40, 20, 16, 8
    n = np.arange(1, N + 1)
    f = np.where(n < Q, np.sin(2 * math.pi * n / 10), np.sin(2 * math.pi * n / 10.5))
    G = hmatrix.hmatrix(f, L, B, T, [1, 2])
    last_before = Q - 1          # 1-based index of the last sample with period 10
    for i in range(N - B + 1):
        for j in range(N - T + 1):
            b_lo, b_hi = i + 1, i + B          # 1-based sample range of the base window
            t_lo, t_hi = j + 1, j + T
            base_side = 0 if b_hi <= last_before else (1 if b_lo > last_before else None)
            test_side = 0 if t_hi <= last_before else (1 if t_lo > last_before else None)
            if base_side is not None and test_side is not None:
                if base_side == test_side:
                    assert abs(G[i, j]) <= 1e-10, (i, j)
                else:
                    assert G[i, j] > 1e-4, (i, j)


def test_rejects_bad_parameters():
    f = _sine(50, 10)
    with pytest.raises(ValueError):
        hmatrix.hmatrix(f, 10, 10, 20, [1])     # B must exceed L
    with pytest.raises(ValueError):
        hmatrix.hmatrix(f, 10, 20, 9, [1])      # T >= L
    with pytest.raises(ValueError):
        hmatrix.hmatrix(f, 10, 20, 20, [0])     # 1-based indices
