"""Pins for the oracle's trajectory matrix, fast matvecs (Algorithms 2/3) and
Hankelization (section 2.4, Algorithm 4)."""
import numpy as np
import pytest

from oracle import fast_hankel, trajectory
from paper_0911_4498_gb300 import synth


def test_trajectory_matrix_matches_display(golden):
    g = golden("trajectory_f1to7_L3.txt")
    X = trajectory.trajectory_matrix(g["f"], int(g["L"][0]))
    np.testing.assert_array_equal(X, np.array(g["row"]))


def test_diagonal_average_hand_examples(golden):
    g = golden("diagonal_average_hand.txt")
    np.testing.assert_allclose(trajectory.diagonal_average(np.array(g["caseA_row"])), g["caseA_g"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(trajectory.diagonal_average(np.array(g["caseB_row"])), g["caseB_g"], rtol=0, atol=1e-15)
    # L > K: the antidiagonals of Y^T are those of Y
    np.testing.assert_allclose(trajectory.diagonal_average(np.array(g["caseA_row"]).T), g["caseA_g"], atol=1e-15)


def test_counts_match_algorithm4_weights(golden):
    g = golden("hankel_counts.txt")
    np.testing.assert_array_equal(trajectory.antidiagonal_counts(int(g["N"][0]), int(g["L"][0])), g["w"])
    np.testing.assert_array_equal(trajectory.antidiagonal_counts(int(g["N2"][0]), int(g["L2"][0])), g["w2"])
    # counts are symmetric in L <-> K
    for N, L in [(10, 3), (10, 8), (11, 6)]:
        np.testing.assert_array_equal(trajectory.antidiagonal_counts(N, L), trajectory.antidiagonal_counts(N, N - L + 1))


def test_circulant_column(golden):
    g = golden("circulant_column.txt")
    f, L = g["f"], int(g["L"][0])
    np.testing.assert_array_equal(fast_hankel.circulant_column(f, L, 5), g["c_M5"])
    np.testing.assert_array_equal(fast_hankel.circulant_column(f, L, 8), g["c_M8"])


def test_hankelize_trajectory_returns_series():
    f = synth.three_sines(200, seed=5)
    for L in [2, 37, 100, 150, 199]:
        np.testing.assert_allclose(trajectory.diagonal_average(trajectory.trajectory_matrix(f, L)), f, rtol=0, atol=1e-14)


def _pow2_at_least(n):
    m = 1
    while m < n:
        m *= 2
    return m


@pytest.mark.parametrize("N", [3, 4, 5, 17, 64, 100, 255])
def test_fast_matvecs_match_explicit_X_all_L(N):
    rng = np.random.default_rng(N)
    f = rng.standard_normal(N)
    for L in range(2, N):
        K = N - L + 1
        X = trajectory.trajectory_matrix(f, L)
        v = rng.standard_normal(K)
        u = rng.standard_normal(L)
        scale = np.abs(X).sum()
        for M in sorted({_pow2_at_least(N), _pow2_at_least(2 * N), _pow2_at_least(N + 3)}):
            ch = fast_hankel.spectrum(f, L, M)
            p = fast_hankel.hankel_matvec(ch, N, L, v)
            q = fast_hankel.hankel_rmatvec(ch, N, L, u)
            assert np.max(np.abs(p - X @ v)) <= 1e-13 * scale
            assert np.max(np.abs(q - X.T @ u)) <= 1e-13 * scale


def test_adjointness_and_M_independence():
    N, L = 1000, 400
    K = N - L + 1
    rng = np.random.default_rng(7)
    f = synth.three_sines(N, seed=3)
    u = rng.standard_normal(L)
    v = rng.standard_normal(K)
    outs = []
    for M in [1024, 2048, 4096]:
        ch = fast_hankel.spectrum(f, L, M)
        Xv = fast_hankel.hankel_matvec(ch, N, L, v)
        Xtu = fast_hankel.hankel_rmatvec(ch, N, L, u)
        assert abs(u @ Xv - Xtu @ v) <= 1e-12 * np.abs(u).sum() * np.abs(Xv).max() * 10
        outs.append((Xv, Xtu))
    for Xv, Xtu in outs[1:]:
        np.testing.assert_allclose(Xv, outs[0][0], atol=1e-11)
        np.testing.assert_allclose(Xtu, outs[0][1], atol=1e-11)


@pytest.mark.parametrize("N,L", [(5, 2), (20, 7), (64, 32), (257, 100), (512, 256), (300, 280)])
def test_rank1_hankelization_matches_naive(N, L):
    K = N - L + 1
    rng = np.random.default_rng(N + L)
    u = rng.standard_normal(L)
    v = rng.standard_normal(K)
    s = 2.5
    naive = trajectory.diagonal_average(s * np.outer(u, v))
    for M in [None, _pow2_at_least(N), _pow2_at_least(4 * N)]:
        got = fast_hankel.rank1_hankelization(s, u, v, M)
        assert np.max(np.abs(got - naive)) <= 1e-13 * s * np.abs(u).max() * np.abs(v).max() * min(L, K)


def test_hankelization_linearity_and_exact_rank1():
    N, L = 300, 120
    K = N - L + 1
    rng = np.random.default_rng(3)
    u1, u2 = rng.standard_normal(L), rng.standard_normal(L)
    v1, v2 = rng.standard_normal(K), rng.standard_normal(K)
    a = fast_hankel.rank1_hankelization(1.5, u1, v1) + fast_hankel.rank1_hankelization(-0.5, u2, v2)
    b = trajectory.diagonal_average(1.5 * np.outer(u1, v1) - 0.5 * np.outer(u2, v2))
    np.testing.assert_allclose(a, b, atol=1e-12)
    # a geometric series is rank 1: X = a x y^T; Hankelizing it returns f
    q = 0.99
    f = synth.geometric(N, q)
    x = q ** np.arange(L)
    y = q ** np.arange(K)
    np.testing.assert_allclose(fast_hankel.rank1_hankelization(q, x, y), f, rtol=1e-13)
