"""Pins for the oracle's SVD of the trajectory matrix (section 2.2) against closed forms,
an independent library SVD, the Frobenius identity and exact reconstruction."""
import math

import numpy as np
import pytest

from oracle import jacobi, ssa, trajectory
from paper_0911_4498_gb300 import synth


def _subspace_sin(A, B):
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return math.sqrt(max(0.0, 1.0 - float(np.min(s)) ** 2))


@pytest.mark.parametrize("shape", [(1, 1), (5, 3), (3, 5), (40, 40), (60, 25), (120, 121)])
def test_jacobi_matches_library_svd(shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    U, s, V = jacobi.svd(A)
    s_ref = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(s, s_ref, rtol=1e-13, atol=1e-13 * s_ref[0])
    np.testing.assert_allclose((U * s) @ V.T, A, atol=1e-13 * s_ref[0])
    r = min(shape)
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-13)


def test_geometric_series_closed_form():
    for a, N, L in [(0.97, 60, 25), (1.01, 80, 40), (-0.9, 41, 20)]:
        f = synth.geometric(N, a)
        K = N - L + 1
        x = a ** np.arange(L)
        y = a ** np.arange(K)
        sig1 = abs(a) * np.linalg.norm(x) * np.linalg.norm(y)
        out = ssa.decompose(f, L, min(L, K), method="jacobi")
        assert abs(out["sigma"][0] - sig1) <= 1e-13 * sig1
        assert np.all(out["sigma"][1:] <= 1e-13 * sig1)
        assert abs(abs(out["U"][:, 0] @ x) / np.linalg.norm(x) - 1) <= 1e-13
        assert abs(abs(out["V"][:, 0] @ y) / np.linalg.norm(y) - 1) <= 1e-13
        # Hankelizing sigma_1 u_1 v_1^T returns f exactly
        rec = ssa.reconstruct(N, L, out["sigma"], out["U"], out["V"], [[0]])[0]
        np.testing.assert_allclose(rec, f, atol=1e-13 * np.abs(f).max())


def test_periodic_cosine_closed_form():
    T, L, K, A = 10, 50, 60, 3.0
    N = L + K - 1
    f = synth.cosine(N, T, A, phi=0.7)
    out = ssa.decompose(f, L, 4, method="jacobi")
    want = A * math.sqrt(L * K) / 2
    np.testing.assert_allclose(out["sigma"][:2], [want, want], rtol=1e-13)
    assert np.all(out["sigma"][2:] <= 1e-12 * want)


def test_frobenius_identity_and_full_reconstruction():
    N, L = 120, 45
    f = synth.three_sines(N, seed=9)
    K = N - L + 1
    out = ssa.decompose(f, L, min(L, K), method="jacobi")
    frob = np.sum(trajectory.antidiagonal_counts(N, L) * f * f)
    assert abs(np.sum(out["sigma"] ** 2) - frob) <= 1e-12 * frob
    # each elementary component on its own, summed, gives f back (sections 2.3-2.4)
    comps = ssa.reconstruct(N, L, out["sigma"], out["U"], out["V"], [[i] for i in range(min(L, K))])
    np.testing.assert_allclose(comps.sum(axis=0), f, atol=1e-12 * np.abs(f).max())
    fftc = ssa.reconstruct(N, L, out["sigma"], out["U"], out["V"], [[0, 1], [2, 3, 4]], method="fft")
    naive = ssa.reconstruct(N, L, out["sigma"], out["U"], out["V"], [[0, 1], [2, 3, 4]], method="naive")
    np.testing.assert_allclose(fftc, naive, atol=1e-12 * np.abs(f).max())


def test_finite_rank_series_reconstructs_exactly():
    N, L = 200, 80
    f = synth.cosine(N, 20, 2.0, 0.1) + synth.geometric(N, 0.995)  # rank 3
    out = ssa.decompose(f, L, 3, method="jacobi")
    rec = ssa.reconstruct(N, L, out["sigma"], out["U"], out["V"], [[0, 1, 2]])[0]
    np.testing.assert_allclose(rec, f, atol=1e-11 * np.abs(f).max())


def test_sign_rule_and_L_greater_than_K():
    N = 90
    f = synth.three_sines(N, seed=2)
    a = ssa.decompose(f, 30, 5, method="jacobi")
    b = ssa.decompose(f, 61, 5, method="jacobi")   # K = 30: X_61 = X_30^T
    np.testing.assert_allclose(a["sigma"], b["sigma"], rtol=1e-13)
    for i in range(5):
        u = a["U"][:, i]
        assert u[np.argmax(np.abs(u))] > 0
        assert abs(abs(a["U"][:, i] @ b["V"][:, i]) - 1) < 1e-10
    with pytest.raises(ValueError):
        ssa.decompose(f, 1, 2)
    with pytest.raises(ValueError):
        ssa.decompose(f, 30, 31 + 40)
