"""GPU parity of the spectral kernels against the oracle: the cached spectrum
(Algorithm 2 steps 1-2), X v and X^T u (Algorithms 2 and 3), batched products,
and grouped Hankelization (Algorithm 4), on the single-CTA and four-step paths."""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import fast_hankel, trajectory
from paper_0911_4498_gb300 import synth
from ssa_testlib import gpu_hankelize, gpu_matvec, gpu_spectrum

pytestmark = pytest.mark.gpu

# FP64-class (double-float) products: normwise error ~ 48-bit rounding x log M
TOL_F64 = 2e-13
TOL_F32C = 3e-6


def _scale(f, x):
    return np.linalg.norm(f) * np.linalg.norm(x)


@pytest.mark.parametrize("N,L", [(3, 2), (5, 3), (17, 5), (100, 50), (1000, 500), (1023, 300), (1025, 1000),
                                 (4097, 2048), (16385, 8000), (40000, 13333)])
def test_spectrum_matches_oracle_fft(N, L):
    f = synth.three_sines(N, seed=N)
    got, M, _ = gpu_spectrum(f, L)
    Lw = min(L, N - L + 1)
    ref = fast_hankel.spectrum(f, Lw, M)[: M // 2 + 1]
    assert np.max(np.abs(got - ref)) <= TOL_F64 * np.max(np.abs(ref)) * 10


SIZES = [(3, 2), (4, 2), (5, 4), (17, 9), (64, 2), (100, 63), (257, 128), (1000, 500), (1000, 999), (2048, 1024)]


@pytest.mark.parametrize("N,L", SIZES)
@pytest.mark.parametrize("prec", [ssa.SSA_PREC_F64, ssa.SSA_PREC_F32C])
def test_matvec_matches_explicit_X(N, L, prec):
    rng = np.random.default_rng(N * 7 + L)
    f = rng.standard_normal(N)
    K = N - L + 1
    X = trajectory.trajectory_matrix(f, L)
    tol = TOL_F64 if prec == ssa.SSA_PREC_F64 else TOL_F32C
    v = rng.standard_normal((3, K))
    u = rng.standard_normal((3, L))
    Xv = gpu_matvec(f, L, v, 0, prec)
    Xtu = gpu_matvec(f, L, u, 1, prec)
    for j in range(3):
        assert np.max(np.abs(Xv[j] - X @ v[j])) <= tol * _scale(f, v[j])
        assert np.max(np.abs(Xtu[j] - X.T @ u[j])) <= tol * _scale(f, u[j])


@pytest.mark.parametrize("N,L", [(8193, 4096), (16384, 8192), (16385, 5000), (32768, 30000), (65536, 32768),
                                 (262147, 131000)])
@pytest.mark.parametrize("prec", [ssa.SSA_PREC_F64, ssa.SSA_PREC_F32C])
def test_matvec_large_matches_oracle(N, L, prec):
    rng = np.random.default_rng(N + L)
    f = synth.many_sines(N, seed=5)
    K = N - L + 1
    M = fast_hankel.fft_length(N)
    Lw = min(L, K)
    ch = fast_hankel.spectrum(f, Lw, M)
    tol = TOL_F64 if prec == ssa.SSA_PREC_F64 else TOL_F32C
    v = rng.standard_normal((2, K))
    u = rng.standard_normal((2, L))
    Xv = gpu_matvec(f, L, v, 0, prec)
    Xtu = gpu_matvec(f, L, u, 1, prec)
    for j in range(2):
        if L <= K:
            rv = fast_hankel.hankel_matvec(ch, N, L, v[j])
            ru = fast_hankel.hankel_rmatvec(ch, N, L, u[j])
        else:  # X = (K-window matrix)^T
            rv = fast_hankel.hankel_rmatvec(ch, N, K, v[j])
            ru = fast_hankel.hankel_matvec(ch, N, K, u[j])
        assert np.max(np.abs(Xv[j] - rv)) <= tol * _scale(f, v[j])
        assert np.max(np.abs(Xtu[j] - ru)) <= tol * _scale(f, u[j])
    # sampled rows by the definition X[i, :] . v = sum_m f[i+m] v[m]
    for i in [0, 1, L // 2, L - 1]:
        assert abs(Xv[0][i] - f[i:i + K] @ v[0]) <= tol * _scale(f, v[0])


def test_matvec_adjointness_full_size():
    N, L = 1 << 20, 1 << 19
    K = N - L + 1
    f = synth.many_sines(N, seed=1)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(L)
    v = rng.standard_normal(K)
    Xv = gpu_matvec(f, L, v, 0)[0]
    Xtu = gpu_matvec(f, L, u, 1)[0]
    assert abs(u @ Xv - Xtu @ v) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(Xv) * 10
    for i in [0, 12345, L - 1]:
        assert abs(Xv[i] - f[i:i + K] @ v) <= TOL_F64 * _scale(f, v)
    for j in [0, 777, K - 1]:
        assert abs(Xtu[j] - f[j:j + L] @ u) <= TOL_F64 * _scale(f, u)


@pytest.mark.parametrize("N,L", [(3, 2), (20, 7), (300, 120), (300, 250), (1000, 500), (8193, 4000),
                                 (20000, 6667)])
@pytest.mark.parametrize("prec", [ssa.SSA_PREC_F64, ssa.SSA_PREC_F32C])
def test_hankelize_matches_oracle(N, L, prec):
    K = N - L + 1
    rng = np.random.default_rng(N)
    r = 5
    sigma = np.abs(rng.standard_normal(r)) * 10 + 1
    U = rng.standard_normal((L, r)) / np.sqrt(L)
    V = rng.standard_normal((K, r)) / np.sqrt(K)
    # groups of two, one and no members: at the four-step sizes the components go in rounds
    # (round r: the r-th member of every group) and an empty group reconstructs to zero
    groups = [[0, 2], [1], [], [4, 3]]
    got = gpu_hankelize(N, L, sigma, U, V, groups, prec)
    tol = 1e-12 if prec == ssa.SSA_PREC_F64 else 2e-6
    assert np.all(got[2] == 0.0)
    for g, idx in enumerate(groups):
        if not idx:
            continue
        if N <= 1000:
            ref = trajectory.diagonal_average((U[:, idx] * sigma[idx]) @ V[:, idx].T)
        else:
            ref = sum(fast_hankel.rank1_hankelization(sigma[i], U[:, i], V[:, i]) for i in idx)
        scale = np.max(sigma) * np.max(np.abs(U)) * np.max(np.abs(V)) * len(idx)
        assert np.max(np.abs(got[g] - ref)) <= tol * scale


def test_invalid_arguments_are_rejected():
    with pytest.raises(ssa.SSAError):
        ssa.ssa_embed_plan(2, 1)
    with pytest.raises(ssa.SSAError):
        ssa.ssa_embed_plan(100, 100)
    plan = ssa.ssa_embed_plan(100, 40)
    try:
        with pytest.raises(ssa.SSAError):
            ssa.ssa_matvec(plan, 0, np.zeros(61), np.zeros(40), 1)   # no series yet
        f = np.ones(100)
        f[3] = np.nan
        with pytest.raises(ssa.SSAError):
            ssa.ssa_set_series(plan, f)
        ssa.ssa_set_series(plan, np.ones(100))
        off, idx = ssa.groups_csr([[0, 1], [1]])
        with pytest.raises(ssa.SSAError):   # overlapping groups
            ssa.ssa_hankelize(plan, np.ones(2), np.ones(80), 40, np.ones(122), 61, 2, off, idx, 2, np.zeros(200))
    finally:
        ssa.ssa_plan_destroy(plan)


def test_fourstep_autotuner_picks_a_tiling_and_results_match():
    """A plan with the four-step path tunes the column tiling once; products
    with the tuned tiling match the oracle like any other."""
    ssa_mod = ssa
    N, L = 300001, 100000
    for prec, tol in ((ssa_mod.SSA_PREC_F64, 1e-12), (ssa_mod.SSA_PREC_F32C, 1e-5)):
        f = synth.three_sines(N, seed=11)
        x = np.random.default_rng(1).standard_normal(N - L + 1)
        y = gpu_matvec(f, L, x, transpose=False, precision=prec)
        fw, inv = ssa_mod.ssa_fft_tiling(prec, N)
        assert fw >= 1 and inv >= 1 and (fw & (fw - 1)) == 0 and (inv & (inv - 1)) == 0
        tf, tr, ti = ssa_mod.ssa_fft_threads(prec, N)
        assert tf in (128, 256, 512) and ti in (128, 256, 512) and tr in (256, 512)
        M = fast_hankel.fft_length(N)
        ref = fast_hankel.hankel_matvec(fast_hankel.spectrum(f, L, M), N, L, x)
        assert np.max(np.abs(y - ref)) <= tol * np.max(np.abs(ref))
