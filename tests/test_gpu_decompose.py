"""GPU parity of the whole decomposition (GKL with CGS2, thick restart, projected
SVD, Ritz vectors, sign rule) and of ssa_reconstruct, against the oracle and
closed forms."""
import math

import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import ssa as ossa
from oracle import trajectory
from paper_0911_4498_gb300 import synth
from ssa_testlib import compare_vectors, gpu_decompose, gpu_decompose_reconstruct

from conftest import load_golden

pytestmark = pytest.mark.gpu

SIG_F64 = 1e-10     # sigma relative error, FP64-class path
REC_F64 = 1e-9      # reconstruction relative L2 error
SIG_F32C = 1e-5


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


def test_three_sines_N1000_full_pipeline():
    N, L, k = 1000, 500, 10
    f = synth.three_sines(N, seed=0)
    ref = ossa.decompose(f, L, k, method="jacobi")
    groups = [[i] for i in range(k)]
    got = gpu_decompose_reconstruct(f, L, k, groups)
    assert got["rc"] == ssa.SSA_OK and got["info"]["converged"]
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F64
    compare_vectors(got["U"], ref["U"], ref["sigma"], 1e-8)
    compare_vectors(got["V"], ref["V"], ref["sigma"], 1e-8)
    rec_ref = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], groups)
    for g in range(k):
        err = np.linalg.norm(got["rec"][g] - rec_ref[g]) / np.linalg.norm(rec_ref[g])
        assert err <= REC_F64, (g, err)
    # the GPU's own triples Hankelize (through the oracle) to the same series
    rec_own = ossa.reconstruct(N, L, got["sigma"], got["U"], got["V"], groups)
    assert np.max(np.abs(rec_own - got["rec"])) <= 1e-11 * np.abs(f).max()
    # sign rule
    for i in range(k):
        u = got["U"][:, i]
        assert u[np.argmax(np.abs(u))] > 0


@pytest.mark.parametrize("N,L,k", [(37, 12, 3), (129, 64, 5), (257, 100, 8), (500, 250, 8), (777, 300, 12),
                                   (2049, 1024, 6), (5000, 1667, 10)])
def test_ragged_sizes_match_oracle(N, L, k):
    f = synth.three_sines(N, seed=N)
    ref = ossa.decompose(f, L, k, method="jacobi" if N <= 1500 else "lanczos")
    got = gpu_decompose(f, L, k)
    assert got["rc"] == ssa.SSA_OK
    assert np.max(np.abs(got["sigma"] - ref["sigma"]) / ref["sigma"]) <= SIG_F64
    compare_vectors(got["U"], ref["U"], ref["sigma"], 1e-7)


def test_window_larger_than_K():
    f = synth.three_sines(600, seed=8)
    ref = ossa.decompose(f, 450, 6, method="jacobi")
    got = gpu_decompose(f, 450, 6)
    assert got["U"].shape == (450, 6) and got["V"].shape == (151, 6)
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F64
    compare_vectors(got["U"], ref["U"], ref["sigma"], 1e-8)
    compare_vectors(got["V"], ref["V"], ref["sigma"], 1e-8)


def test_geometric_series_rank_one_breakdown():
    N, L, a = 300, 120, 0.99
    K = N - L + 1
    f = synth.geometric(N, a)
    x = a ** np.arange(L)
    y = a ** np.arange(K)
    s1 = a * np.linalg.norm(x) * np.linalg.norm(y)
    got = gpu_decompose(f, L, 4)
    assert got["rc"] == ssa.SSA_OK
    assert abs(got["sigma"][0] - s1) <= 1e-12 * s1
    assert np.all(np.abs(got["sigma"][1:]) <= 1e-12 * s1)
    assert abs(abs(got["U"][:, 0] @ x) / np.linalg.norm(x) - 1) <= 1e-12


def test_periodic_cosine_rank_two():
    T, L, K, A = 10, 50, 60, 3.0
    N = L + K - 1
    f = synth.cosine(N, T, A, 0.7)
    got = gpu_decompose(f, L, 3)
    want = A * math.sqrt(L * K) / 2
    np.testing.assert_allclose(got["sigma"][:2], [want, want], rtol=1e-12)
    assert got["sigma"][2] <= 1e-12 * want


def test_zero_series():
    got = gpu_decompose(np.zeros(64), 20, 3)
    assert np.all(got["sigma"] == 0.0)


def test_full_rank_request_and_frobenius():
    N, L = 60, 20
    f = synth.three_sines(N, seed=4)
    got = gpu_decompose(f, L, L)
    frob = np.sum(trajectory.antidiagonal_counts(N, L) * f * f)
    assert abs(np.sum(got["sigma"] ** 2) - frob) <= 1e-11 * frob


def test_two_seeds_agree():
    f = synth.three_sines(1000, seed=0)
    a = gpu_decompose(f, 500, 10, seed=1)
    b = gpu_decompose(f, 500, 10, seed=2)
    assert np.max(_rel(a["sigma"], b["sigma"])) <= SIG_F64


def test_f32c_precision_mode():
    N, L, k = 1000, 500, 10
    f = synth.three_sines(N, seed=0)
    ref = ossa.decompose(f, L, k, method="jacobi")
    got = gpu_decompose(f, L, k, precision=ssa.SSA_PREC_F32C)
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F32C


def test_bad_k_rejected():
    with pytest.raises(ssa.SSAError):
        gpu_decompose(synth.three_sines(100, 1), 40, 41)
    with pytest.raises(ssa.SSAError):
        gpu_decompose(synth.three_sines(100, 1), 40, 0)


@pytest.mark.parametrize("N,L,k", [(5000, 2500, 16), (40000, 13333, 12)])
def test_rayleigh_refinement(N, L, k):
    """With refinement each sigma_i is u_i^T X v_i of the returned vectors,
    computed with native-FP64 products: one CTA (n <= 8192) and four-step
    (n = 32768) products, F64 and F32C; values stay sorted and within the
    precision's tolerance; k extra products are counted."""
    from oracle import fast_hankel
    f = synth.many_sines(N, seed=3)
    ref = ossa.decompose(f, L, k, method="lanczos")
    for prec, tol in ((ssa.SSA_PREC_F64, SIG_F64), (ssa.SSA_PREC_F32C, SIG_F32C)):
        got = gpu_decompose(f, L, k, precision=prec, refine=ssa.SSA_REFINE_ON)
        chat = fast_hankel.spectrum(f, L, fast_hankel.fft_length(N))
        XV = np.stack([fast_hankel.hankel_matvec(chat, N, L, got["V"][:, i]) for i in range(k)], axis=1)
        rq = np.einsum("ij,ij->j", got["U"], XV)
        assert np.max(np.abs(got["sigma"] - rq)) <= 1e-12 * got["sigma"][0], prec
        assert np.max(_rel(got["sigma"], ref["sigma"])) <= tol, prec
        assert np.all(np.diff(got["sigma"]) <= 0)
    off = gpu_decompose(f, L, k)
    on = gpu_decompose(f, L, k, refine=ssa.SSA_REFINE_ON)
    assert on["info"]["matvecs"] == off["info"]["matvecs"] + k
    assert np.max(_rel(off["sigma"], on["sigma"])) <= SIG_F64


def test_bad_refine_mode_rejected():
    with pytest.raises(ssa.SSAError):
        gpu_decompose(synth.three_sines(100, 1), 40, 3, refine=7)


@pytest.fixture(scope="module")
def unit_refs():
    """Oracle decompositions of the unscaled series (computed once)."""
    from oracle import fast_hankel
    out = {}
    for N, L, k in ((1000, 500, 10), (40000, 13000, 8)):
        f0 = synth.three_sines(N, seed=N + 1)
        ref = ossa.decompose(f0, L, k, method="jacobi" if N <= 1500 else "lanczos")
        chat = fast_hankel.spectrum(f0, L, fast_hankel.fft_length(N), "library")
        out[N] = (f0, L, k, ref, chat)
    for n in (800, 3000):
        f0 = synth.three_sines(n, seed=n)
        out[("batch", n)] = (f0, ossa.decompose(f0, n // 2, 6, method="jacobi" if n <= 1500 else "lanczos"))
    return out


@pytest.mark.parametrize("scale", [1e25, 1e-25, 1e200, 1e-200])
def test_series_units_do_not_matter(unit_refs, scale):
    """Double-float has FP32's exponent range; the library holds the series
    scaled by an exact power of two, so sigma, products and reconstructions of
    a series in any units are the unscaled ones times the scale (against the
    oracle, sigma <= 1e-10, reconstruction <= 1e-9, for a single-CTA and a
    four-step plan, and in the batched engine)."""
    from oracle import fast_hankel
    from ssa_testlib import gpu_matvec
    for N in (1000, 40000):
        f0, L, k, ref, chat = unit_refs[N]
        f = f0 * scale
        groups = [[0, 1], [2, 3]]
        got = gpu_decompose_reconstruct(f, L, k, groups)
        assert got["rc"] == ssa.SSA_OK
        assert np.max(_rel(got["sigma"], ref["sigma"] * scale)) <= SIG_F64
        # compared in the series' own units (a norm of 1e200-sized values overflows)
        rec_ref = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], groups, method="fft", fft="library")
        for g in range(len(groups)):
            err = np.linalg.norm(got["rec"][g] / scale - rec_ref[g]) / np.linalg.norm(rec_ref[g])
            assert err <= REC_F64, (N, g, err)
        # a product of the scaled series is the scaled product
        K = N - L + 1
        x = np.random.default_rng(3).standard_normal(K)
        y = gpu_matvec(f, L, x, 0)[0]
        want = fast_hankel.hankel_matvec(chat, N, L, x, "library")
        assert np.max(np.abs(y / scale - want)) <= 1e-13 * np.linalg.norm(f0) * np.linalg.norm(x)
    # batched engine (one persistent launch), per-series scaling
    f_a, r_a = unit_refs[("batch", 800)]
    f_b, r_b = unit_refs[("batch", 3000)]
    flat = np.concatenate([f_a, f_b]) * scale
    off = np.array([0, 800, 3800], dtype=np.int64)
    b, rc = ssa.ssa_decompose_batch(flat, off, np.array([400, 1500], dtype=np.int64),
                                    np.array([6, 6], dtype=np.int32), ssa.make_opts())
    try:
        for j, r in enumerate((r_a, r_b)):
            sig = np.empty(6)
            ssa.ssa_batch_get(b, j, sig)
            assert np.max(_rel(sig, r["sigma"] * scale)) <= SIG_F64
    finally:
        ssa.ssa_batch_destroy(b)


def test_reorth_skip_option():
    """The skip test of the reorthogonalisation (opt-in level tau): sigma within 1e-10 of the
    oracle on a well-separated spectrum, in the single-series and the batched engine; out of
    range levels are rejected; F32C ignores it (one pass already)."""
    N, L, k = 5000, 2500, 16
    f = synth.many_sines(N, seed=11)
    ref = ossa.decompose(f, L, k, method="lanczos")
    got = gpu_decompose(f, L, k, reorth_skip=1e-12)
    assert got["rc"] == ssa.SSA_OK
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F64
    compare_vectors(got["U"], ref["U"], ref["sigma"], 1e-9, res_tol=1e-11)
    b, rc = ssa.ssa_decompose_batch(f, np.array([0, N], dtype=np.int64), np.array([L], dtype=np.int64),
                                    np.array([k], dtype=np.int32), ssa.make_opts(reorth_skip=1e-12))
    try:
        sig = np.empty(k)
        ssa.ssa_batch_get(b, 0, sig)
        assert np.max(_rel(sig, ref["sigma"])) <= SIG_F64
    finally:
        ssa.ssa_batch_destroy(b)
    for bad in (-1.0, 0.5):
        with pytest.raises(ssa.SSAError):
            gpu_decompose(f, L, k, reorth_skip=bad)
    f32 = gpu_decompose(f, L, k, precision=ssa.SSA_PREC_F32C, reorth_skip=1e-12)
    assert np.max(_rel(f32["sigma"], ref["sigma"])) <= SIG_F32C


@pytest.mark.parametrize("N,L,k", [(5000, 2500, 16), (40000, 13333, 12)])
def test_partial_reorthogonalisation(N, L, k):
    """PRO (section 3.2.2) where one Lanczos cycle converges (single-CTA and four-step products):
    sigma within 1e-10 of the oracle (their error is second order in the coefficients PRO leaves
    out of B, which are below sqrt(eps) = 2^-23 of the double-float products); vectors within
    sqrt(eps), or Wedin's bound with a residual of 1e-9 sigma_1 where a gap is small; relation (1)
    within 1e-9 sigma_1 and the reconstructions of the leading components within 10 sqrt(eps)."""
    f = synth.many_sines(N, seed=N)
    ref = ossa.decompose(f, L, k, method="lanczos")
    groups = [[0], [1], [2, 3]]
    got = gpu_decompose_reconstruct(f, L, k, groups, reorth=ssa.SSA_REORTH_PRO)
    assert got["rc"] == ssa.SSA_OK and got["info"]["converged"] and got["info"]["restarts"] == 0
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F64
    sqrt_eps = 2.0 ** -23
    compare_vectors(got["U"], ref["U"], ref["sigma"], sqrt_eps, res_tol=1e-9)
    compare_vectors(got["V"], ref["V"], ref["sigma"], sqrt_eps, res_tol=1e-9)
    K = N - L + 1
    for i in (0, k // 2, k - 1):
        for row in (0, L // 3, L - 1):
            lhs = f[row:row + K] @ got["V"][:, i]
            assert abs(lhs - got["sigma"][i] * got["U"][row, i]) <= 1e-9 * ref["sigma"][0]
    rec_ref = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], groups, method="fft", fft="library")
    for gi in range(len(groups)):
        err = np.linalg.norm(got["rec"][gi] - rec_ref[gi]) / np.linalg.norm(rec_ref[gi])
        assert err <= 10 * sqrt_eps, (gi, err)
    with pytest.raises(ssa.SSAError):
        gpu_decompose(f, L, k, reorth=7)


def test_partial_reorthogonalisation_falls_back_to_full():
    """A PRO first cycle that does not converge (N = 5113, k = 100 restarts three times) starts over
    from the same starting vector with full Gram-Schmidt: the result is the full-reorthogonalisation
    result bit for bit, with one more restart counted."""
    N, L, k = 5113, 2556, 100
    f = synth.three_sines(N, seed=7)
    full = gpu_decompose(f, L, k)
    pro = gpu_decompose(f, L, k, reorth=ssa.SSA_REORTH_PRO)
    assert full["rc"] == pro["rc"] == ssa.SSA_OK
    assert full["info"]["restarts"] > 0
    assert pro["info"]["restarts"] == full["info"]["restarts"] + 1
    assert np.array_equal(full["sigma"], pro["sigma"])
    assert np.array_equal(full["U"], pro["U"]) and np.array_equal(full["V"], pro["V"])


@pytest.mark.parametrize("N,L,k,cap,reorth", [(40000, 13333, 12, 16, ssa.SSA_REORTH_FULL),
                                              (65536, 32768, 20, 19, ssa.SSA_REORTH_FULL),
                                              (40000, 13333, 12, 7, ssa.SSA_REORTH_PRO)])
def test_grid_cap(N, L, k, cap, reorth):
    """opts.grid_cap limits the persistent reorthogonalisation passes and the cooperative kernels to
    `cap` CTAs (the server's share per request): the block sums add up in another order, the
    results stay within the FP64 tolerances of the oracle, and a negative cap is rejected."""
    f = synth.many_sines(N, seed=N + cap)
    ref = ossa.decompose(f, L, k, method="lanczos")
    got = gpu_decompose(f, L, k, grid_cap=cap, reorth=reorth)
    assert got["rc"] == ssa.SSA_OK and got["info"]["converged"]
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F64
    tol = 1e-9 if reorth == ssa.SSA_REORTH_FULL else 2.0 ** -23
    compare_vectors(got["U"], ref["U"], ref["sigma"], tol, res_tol=1e-11 if reorth == ssa.SSA_REORTH_FULL else 1e-9)
    with pytest.raises(ssa.SSAError):
        gpu_decompose(f, L, k, grid_cap=-1)


@pytest.mark.parametrize("N,L,k", [(5000, 2500, 8), (5000, 2500, 16), (40000, 13333, 12)])
def test_no_reorthogonalisation_with_ghost_filter(N, L, k):
    """SSA_REORTH_NONE (section 3.2.1): one cycle of 4 x the usual length with no Gram-Schmidt,
    spurious copies removed by the Cullum-Willoughby test.  Where the cycle converges the k
    leading triples, sigma agree with the oracle's to the FP64 tolerance (measured <= 1.5e-14),
    the unit Ritz vectors to 1e-6 (measured <= 2.2e-8: without reorthogonalisation they are
    accurate only as far as the converged copies reach) and the reconstructions of the leading
    components to 1e-8 (measured <= 1.8e-10)."""
    f = synth.many_sines(N, seed=N)
    ref = ossa.decompose(f, L, k, method="lanczos")
    groups = [[0], [1], [2, 3]]
    got = gpu_decompose_reconstruct(f, L, k, groups, reorth=ssa.SSA_REORTH_NONE)
    assert got["rc"] == ssa.SSA_OK and got["info"]["converged"] and got["info"]["restarts"] == 0
    assert got["info"]["krylov_dim"] == 4 * max(2 * k, k + 32)
    assert np.max(_rel(got["sigma"], ref["sigma"])) <= SIG_F64
    compare_vectors(got["U"], ref["U"], ref["sigma"], 1e-6)
    compare_vectors(got["V"], ref["V"], ref["sigma"], 1e-6)
    for Q in (got["U"], got["V"]):
        assert np.max(np.abs(np.linalg.norm(Q, axis=0) - 1.0)) <= 1e-13
    rec_ref = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], groups, method="fft", fft="library")
    for gi in range(len(groups)):
        err = np.linalg.norm(got["rec"][gi] - rec_ref[gi]) / np.linalg.norm(rec_ref[gi])
        assert err <= 1e-8, (gi, err)


def test_no_reorthogonalisation_reports_what_it_misses():
    """k = 100 at N = 5113: the longest cycle allowed (510 steps) does not converge the tail
    without reorthogonalisation; the call returns SSA_ENOCONV with k finite values in descending
    order, the leading ones still right."""
    N, L, k = 5113, 2556, 100
    f = synth.three_sines(N, seed=7)
    got = gpu_decompose(f, L, k, reorth=ssa.SSA_REORTH_NONE)
    assert got["rc"] == ssa.SSA_ENOCONV and not got["info"]["converged"]
    assert got["info"]["krylov_dim"] == 510
    s = got["sigma"]
    assert np.all(np.isfinite(s)) and np.all(np.diff(s) <= 0)
    ref = load_golden("sigma_three_sines_N5113_L2556_k100.txt")["sigma"]
    assert np.max(np.abs(s[:10] - ref[:10]) / ref[:10]) <= SIG_F64
    # the opt-in modes are refused with FP32 products (their error is above sqrt(eps))
    for mode in (ssa.SSA_REORTH_NONE, ssa.SSA_REORTH_PRO):
        with pytest.raises(ssa.SSAError):
            gpu_decompose(f, L, k, precision=ssa.SSA_PREC_F32C, reorth=mode)


@pytest.mark.parametrize("N,L,k,kw", [(40000, 13333, 20, {}), (70000, 35000, 30, {"reorth_skip": 1e-12}),
                                      (5000, 2500, 8, {"reorth": ssa.SSA_REORTH_PRO}), (1000, 500, 10, {})])
def test_repeated_decompositions_replay_cycles_exactly(N, L, k, kw):
    """A plan that decomposes again runs each Lanczos cycle from a CUDA graph (captured on the
    second run of a cycle shape, replayed after): the first, second and third decompositions of
    the same series give the same sigma, vectors and launch count, bit for bit."""
    f = synth.many_sines(N, seed=N + k)
    K = N - L + 1
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(**kw))
    try:
        outs = []
        for _ in range(3):
            l0 = ssa.ssa_kernel_launches()
            d, rc = ssa.ssa_decompose(plan, f, k)
            try:
                sigma, U, V = np.empty(k), np.empty((k, L)), np.empty((k, K))
                ssa.ssa_decomp_get(d, sigma, U, V, None)
                info = ssa.ssa_decomp_info(d)
            finally:
                ssa.ssa_decomp_destroy(d)
            outs.append((rc, sigma, U, V, info, ssa.ssa_kernel_launches() - l0))
        for rc, sigma, U, V, info, nl in outs[1:]:
            assert rc == outs[0][0] == ssa.SSA_OK
            assert np.array_equal(sigma, outs[0][1])
            assert np.array_equal(U, outs[0][2]) and np.array_equal(V, outs[0][3])
            assert info == outs[0][4]
            assert nl == outs[0][5]
    finally:
        ssa.ssa_plan_destroy(plan)
    ref = ossa.decompose(f, L, k, method="jacobi" if N <= 1500 else "lanczos")
    assert np.max(_rel(outs[2][1], ref["sigma"])) <= SIG_F64
