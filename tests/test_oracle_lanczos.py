"""Pins for the oracle's Lanczos SVD (section 3): agreement with the Jacobi oracle,
relation (1), orthogonality, independence of the starting vector, breakdown."""
import numpy as np
import pytest

from oracle import fast_hankel, lanczos, ssa, trajectory
from paper_0911_4498_gb300 import synth


def _match(a, b, k, tol_sigma):
    s1 = a["sigma"][0]
    np.testing.assert_allclose(a["sigma"][:k], b["sigma"][:k], rtol=tol_sigma, atol=tol_sigma * s1)


@pytest.mark.parametrize("N,L,k,seed", [(500, 250, 8, 0), (1000, 500, 10, 0), (777, 300, 12, 4), (1200, 900, 6, 2),
                                        (4000, 500, 10, 3)])
def test_lanczos_matches_jacobi(N, L, k, seed):
    f = synth.three_sines(N, seed=seed)
    a = ssa.decompose(f, L, k, method="jacobi")
    b = ssa.decompose(f, L, k, method="lanczos", seed=11)
    assert b["converged"]
    _match(a, b, k, 1e-12)
    s = a["sigma"]
    for i in range(k):
        gap = min([abs(s[i] - s[j]) for j in range(len(s)) if j != i] + [np.inf]) / s[0]
        if gap > 1e-6:
            assert abs(abs(a["U"][:, i] @ b["U"][:, i]) - 1) < 1e-9
            assert abs(abs(a["V"][:, i] @ b["V"][:, i]) - 1) < 1e-9


def test_two_seeds_agree():
    f = synth.three_sines(1000, seed=0)
    a = ssa.decompose(f, 500, 10, method="lanczos", seed=1)
    b = ssa.decompose(f, 500, 10, method="lanczos", seed=2)
    _match(a, b, 10, 1e-12)


def test_relation1_and_orthogonality():
    N, L, k = 800, 300, 6
    K = N - L + 1
    f = synth.three_sines(N, seed=1)
    M = fast_hankel.fft_length(N)
    ch = fast_hankel.spectrum(f, L, M)
    res = lanczos.gkl_svd(lambda v: fast_hankel.hankel_matvec(ch, N, L, v),
                          lambda u: fast_hankel.hankel_rmatvec(ch, N, L, u), L, K, k, seed=3)
    X = trajectory.trajectory_matrix(f, L)
    s1 = res.sigma[0]
    # A v_i = sigma_i u_i for Ritz triples (from A V = U B), and A^T u_i ~ sigma_i v_i
    assert np.max(np.abs(X @ res.V - res.U * res.sigma)) <= 1e-12 * s1
    assert np.max(np.abs(X.T @ res.U - res.V * res.sigma)) <= 1e-11 * s1
    np.testing.assert_allclose(res.U.T @ res.U, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(res.V.T @ res.V, np.eye(k), atol=1e-13)


def test_breakdown_rank_one_and_rank_two():
    N, L = 300, 120
    f = synth.geometric(N, 0.99)
    out = ssa.decompose(f, L, 4, method="lanczos")
    x = 0.99 ** np.arange(L)
    y = 0.99 ** np.arange(N - L + 1)
    s1 = 0.99 * np.linalg.norm(x) * np.linalg.norm(y)
    assert out["converged"]
    assert abs(out["sigma"][0] - s1) <= 1e-13 * s1
    assert np.all(np.abs(out["sigma"][1:]) <= 1e-12 * s1)
    f2 = synth.cosine(N, 12, 1.5, 0.2)
    out2 = ssa.decompose(f2, L, 3, method="lanczos")
    ref = ssa.decompose(f2, L, 3, method="jacobi")
    np.testing.assert_allclose(out2["sigma"][:2], ref["sigma"][:2], rtol=1e-13)
    assert out2["sigma"][2] <= 1e-12 * ref["sigma"][0]


def test_zero_series_and_full_rank_request():
    out = ssa.decompose(np.zeros(40), 15, 3, method="lanczos")
    assert np.all(out["sigma"] == 0.0)
    f = synth.three_sines(40, seed=1)
    a = ssa.decompose(f, 15, 15, method="lanczos")
    b = ssa.decompose(f, 15, 15, method="jacobi")
    np.testing.assert_allclose(a["sigma"], b["sigma"], rtol=1e-12, atol=1e-12 * b["sigma"][0])


def test_window_larger_than_K():
    f = synth.three_sines(600, seed=8)
    a = ssa.decompose(f, 450, 6, method="lanczos")
    b = ssa.decompose(f, 450, 6, method="jacobi")
    _match(a, b, 6, 1e-12)
    assert a["U"].shape == (450, 6) and a["V"].shape == (151, 6)


def test_library_fft_option_matches_own_fft():
    """The oracle's library-FFT option (used only where its own radix-2 FFT is too slow) gives the
    same products and the same decomposition as its own FFT."""
    f = synth.many_sines(5000, seed=2)
    L, K = 2500, 2501
    M = fast_hankel.fft_length(5000)
    rng = np.random.default_rng(1)
    v, u = rng.standard_normal(K), rng.standard_normal(L)
    c_own, c_lib = fast_hankel.spectrum(f, L, M), fast_hankel.spectrum(f, L, M, "library")
    scale_v, scale_u = np.linalg.norm(f) * np.linalg.norm(v), np.linalg.norm(f) * np.linalg.norm(u)
    assert np.max(np.abs(fast_hankel.hankel_matvec(c_own, 5000, L, v)
                         - fast_hankel.hankel_matvec(c_lib, 5000, L, v, "library"))) <= 1e-13 * scale_v
    assert np.max(np.abs(fast_hankel.hankel_rmatvec(c_own, 5000, L, u)
                         - fast_hankel.hankel_rmatvec(c_lib, 5000, L, u, "library"))) <= 1e-13 * scale_u
    a = ssa.decompose(f, L, 10, method="lanczos", seed=0)
    b = ssa.decompose(f, L, 10, method="lanczos", seed=0, fft="library")
    _match(a, b, 10, 1e-12)
    with pytest.raises(ValueError):
        fast_hankel.spectrum(f, L, M, "other")


def test_library_fft_hankelization_matches_own_fft_and_naive():
    """Algorithm 4 on numpy's FFT (the full-size reconstruction checks use it) equals the oracle's
    own radix-2 FFT and the naive antidiagonal mean of section 2.4, for L <= K and L > K."""
    from oracle import trajectory
    rng = np.random.default_rng(5)
    for N, L in ((300, 120), (301, 200), (4097, 2048)):
        K = N - L + 1
        u, v = rng.standard_normal(L), rng.standard_normal(K)
        own = fast_hankel.rank1_hankelization(1.7, u, v)
        lib = fast_hankel.rank1_hankelization(1.7, u, v, fft="library")
        assert np.max(np.abs(own - lib)) <= 1e-13 * np.max(np.abs(own))
        if N <= 400:
            naive = trajectory.diagonal_average(1.7 * np.outer(u, v))
            assert np.max(np.abs(lib - naive)) <= 1e-13 * np.max(np.abs(naive))
    with pytest.raises(ValueError):
        fast_hankel.rank1_hankelization(1.0, u, v, fft="other")
