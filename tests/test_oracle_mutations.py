"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each test swaps one oracle function for a copy carrying a plausible slip
(the printed off-by-ones of Algorithms 2-4, a sign error, a dropped term)
and checks that the corresponding pin rejects it.
"""
import numpy as np
import pytest

from oracle import dft, fast_hankel, trajectory


def _matvec_pin(f, L):
    N = f.size
    K = N - L + 1
    rng = np.random.default_rng(0)
    v, u = rng.standard_normal(K), rng.standard_normal(L)
    X = trajectory.trajectory_matrix(f, L)
    ch = fast_hankel.spectrum(f, L, 64)
    assert np.allclose(fast_hankel.hankel_matvec(ch, N, L, v), X @ v, atol=1e-10)
    assert np.allclose(fast_hankel.hankel_rmatvec(ch, N, L, u), X.T @ u, atol=1e-10)


def test_alg3_printed_slice_is_caught(monkeypatch):
    def bad_rmatvec(chat, N, L, u):
        M = chat.size
        K = N - L + 1
        w = np.zeros(M)
        w[M - L:] = u[::-1]
        p = dft.ifft_radix2(dft.fft_radix2(w) * chat)
        return p[M - K - 1:M - 1].real            # p'_{L-1}..p'_{N-1}
    f = np.random.default_rng(1).standard_normal(30)
    _matvec_pin(f, 9)
    monkeypatch.setattr(fast_hankel, "hankel_rmatvec", bad_rmatvec)
    with pytest.raises(AssertionError):
        _matvec_pin(f, 9)


def test_case_formula_off_by_one_is_caught(monkeypatch):
    def bad_column(f, L, M):
        N = f.size
        c = np.zeros(M)
        c[:L] = f[N - L:]
        c[L + (M - N):] = np.roll(f[:N - L + 1], -1)[:N - L]   # t_{j-L+1} reading
        return c
    f = np.random.default_rng(2).standard_normal(30)
    monkeypatch.setattr(fast_hankel, "circulant_column", bad_column)
    with pytest.raises(AssertionError):
        _matvec_pin(f, 9)


def test_alg4_multiplying_by_counts_is_caught(monkeypatch):
    N, L = 40, 15
    K = N - L + 1
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(L), rng.standard_normal(K)
    naive = trajectory.diagonal_average(np.outer(u, v))
    orig = fast_hankel.antidiagonal_counts
    monkeypatch.setattr(fast_hankel, "antidiagonal_counts", lambda n, l: 1.0 / orig(n, l))
    assert not np.allclose(fast_hankel.rank1_hankelization(1.0, u, v), naive, atol=1e-8)


def test_fft_sign_error_is_caught(golden):
    g = golden("dft_length4.txt")
    X = dft.fft_radix2(g["x"], inverse=True) * 4     # forward with the wrong sign
    assert not np.allclose(X.imag, g["X_im"])


def test_dropped_count_case_is_caught(golden):
    g = golden("hankel_counts.txt")
    N, L = int(g["N"][0]), int(g["L"][0])
    n = np.arange(N)
    wrong = np.minimum(n + 1, L).astype(float)        # forgets the tail case N-n
    assert not np.array_equal(wrong, g["w"])
    np.testing.assert_array_equal(trajectory.antidiagonal_counts(N, L), g["w"])
