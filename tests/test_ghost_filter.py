"""The Cullum-Willoughby ghost filter of Lanczos without reorthogonalisation (section 3.2.1):
the oracle's filter pinned to the mathematics (a no-reorthogonalisation run on a matrix of known
singular values, whose projected matrix is full of copies and spurious values, filters back to
exactly those values), hand-made cases, and the library's host-side filter (ssa_cw_filter, no GPU
needed) against the oracle's on seeded random inputs."""
import numpy as np
import pytest

from oracle import ghost

TRUE = np.concatenate([np.array([10, 9, 8, 7, 6, 5.5, 5, 4.5]), np.linspace(1.0, 0.1, 52)])


def _matrix():
    rng = np.random.default_rng(3)
    L, K = 80, 60
    Q1, _ = np.linalg.qr(rng.standard_normal((L, L)))
    Q2, _ = np.linalg.qr(rng.standard_normal((K, K)))
    return Q1[:, :K] @ np.diag(TRUE) @ Q2.T


def _run(steps):
    A = _matrix()
    B, alpha_next, U, V = ghost.gkl_no_reorth(lambda x: A @ x, lambda x: A.T @ x, np.ones(A.shape[0]), steps)
    s, res = ghost.ritz_residuals(B, alpha_next)
    s_hat = np.linalg.svd(B[1:, :], compute_uv=False)
    return B, V, s, s_hat, res


@pytest.mark.parametrize("steps", [60, 120])
def test_oracle_recurrence_holds_without_orthogonality(steps):
    """Algorithm 1's two relations hold to rounding however far the vectors have lost orthogonality:
    A V = U B (u-side recurrence) and A^T U_s = V B_s^T (v-side, with B_s the first s rows of B);
    unit-length Lanczos vectors."""
    A = _matrix()
    B, alpha_next, U, V = ghost.gkl_no_reorth(lambda x: A @ x, lambda x: A.T @ x, np.ones(A.shape[0]), steps)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A @ V - U @ B) <= 1e-14 * nA
    assert np.linalg.norm(A.T @ U[:, :steps] - V @ B[:steps, :].T) <= 1e-14 * nA
    assert np.allclose(np.linalg.norm(U, axis=0), 1.0) and np.allclose(np.linalg.norm(V, axis=0), 1.0)
    assert np.max(np.abs(V.T @ V - np.eye(steps))) > 0.5   # while orthogonality is gone


@pytest.mark.parametrize("steps", [60, 90, 120])
def test_oracle_filter_recovers_known_singular_values(steps):
    B, V, s, s_hat, res = _run(steps)
    # the run is deep in the ghost regime: the right vectors have lost orthogonality entirely and
    # sigma(B) holds copies of converged values
    assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) > 0.5
    assert sum(1 for i in range(s.size - 1) if s[i] - s[i + 1] <= 1e-10 * s[0]) >= 10
    keep, ok = ghost.cullum_willoughby(s, s_hat, res, 8, 1e-12)
    assert ok
    assert np.max(np.abs(s[keep] - TRUE[:8]) / TRUE[:8]) <= 1e-12


@pytest.mark.parametrize("steps", [60, 90, 120])
def test_oracle_filter_without_the_comparison_keeps_a_spurious_value(steps):
    """A filter that skipped the comparison with B without its first row would keep a spurious
    simple value among the leading eight (the pin above would then fail)."""
    B, V, s, s_hat, res = _run(steps)
    keep, _ = ghost.cullum_willoughby(s, np.array([]), res, 8, 1e-12)
    assert np.max(np.abs(s[keep] - TRUE[:8]) / TRUE[:8]) > 1e-3


def test_oracle_filter_hand_cases():
    r = np.full(6, 1e-20)
    # copies kept once (smallest residual), a simple value present in sigma_hat dropped
    keep, ok = ghost.cullum_willoughby([5, 4, 4, 3, 2, 1], [4.5, 3, 1.5], [1e-20, 1e-20, 1e-18, 1e-20, 1e-20, 1e-20], 3,
                                       1e-12)
    assert keep == [0, 1, 4] and ok
    keep, ok = ghost.cullum_willoughby([5, 4, 4, 3, 2, 1], [4.5, 3, 1.5], [1e-20, 1e-18, 1e-20, 1e-20, 1e-20, 1e-20], 3,
                                       1e-12)
    assert keep == [0, 2, 4] and ok
    # copies stay genuine even when sigma_hat holds the value too
    keep, ok = ghost.cullum_willoughby([5, 4, 4, 3], [4], r[:4], 2, 1e-12)
    assert keep == [0, 1] and ok
    # fewer than k pass: padded with the largest unused indices, not converged
    keep, ok = ghost.cullum_willoughby([5, 4, 3], [5, 4], r[:3], 2, 1e-12)
    assert keep == [0, 2] and not ok
    # a kept value whose residual is above tol sigma_1: not converged
    keep, ok = ghost.cullum_willoughby([5, 4, 3], [], [1e-20, 1e-9, 1e-20], 2, 1e-12)
    assert keep == [0, 1] and not ok
    # values at or below the agreement level are not candidates
    keep, ok = ghost.cullum_willoughby([1.0, 1e-12, 1e-13], [], r[:3], 2, 1e-12)
    assert keep == [0, 1] and not ok


def _random_case(rng):
    c = int(rng.integers(1, 40))
    base = np.sort(rng.uniform(0.01, 1.0, c))[::-1]
    s = []
    for v in base:  # some values repeated (copies) within the agreement level
        s.append(v)
        if rng.random() < 0.3:
            s.append(v * (1 - rng.uniform(0, 5e-11)))
    s = np.sort(np.array(s))[::-1]
    hat = [v * (1 + rng.uniform(-5e-11, 5e-11)) for v in s if rng.random() < 0.3]
    hat += list(rng.uniform(0.0, 1.0, int(rng.integers(0, 5))))
    res = 10.0 ** rng.uniform(-18, -9, s.size)
    k = int(rng.integers(1, s.size + 1))
    return s, np.array(hat), res, k


@pytest.fixture(scope="module")
def built():
    from paper_0911_4498_gb300 import build
    return build.build()


def test_library_filter_matches_oracle(built):
    import paper_0911_4498_gb300 as ssa
    rng = np.random.default_rng(11)
    for _ in range(300):
        s, hat, res, k = _random_case(rng)
        keep_lib, ok_lib = ssa.ssa_cw_filter(s, hat, res, k, 1e-12)
        keep_or, ok_or = ghost.cullum_willoughby(s, hat, res, k, 1e-12)
        assert list(keep_lib) == keep_or and ok_lib == ok_or, (s, hat, res, k)


def test_library_filter_rejects_bad_input(built):
    import paper_0911_4498_gb300 as ssa
    s = np.array([3.0, 2.0, 1.0])
    with pytest.raises(ssa.SSAError):
        ssa.ssa_cw_filter(s, np.array([]), np.zeros(3), 4, 1e-12)
    with pytest.raises(ssa.SSAError):
        ssa.ssa_cw_filter(s[::-1].copy(), np.array([]), np.zeros(3), 2, 1e-12)
    with pytest.raises(ssa.SSAError):
        ssa.ssa_cw_filter(np.array([3.0, np.nan]), np.array([]), np.zeros(2), 1, 1e-12)
