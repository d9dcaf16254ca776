"""GPU parity at the sizes whose expected values the oracle wrote ahead of time
(tests/golden, by make_golden.py from the oracle only), and at Krylov
dimensions above 256 against the Jacobi oracle.

  * N = 5113, L = 2556, k = 100 (shape of the section 7 monthly-births run):
    d = 200, so the projected SVD runs the cluster kernels with eight column
    pieces per lane;
  * N = 2^22, L = 2^21, k = 100, exact-rank-40 damped cosines + N(0, 1e-6^2)
    (the precision-stress workload), both precisions: per-sigma errors on the
    signal triples, |d sigma_i| / sigma_1 on the noise bulk, sampled vector
    entries, and the reconstruction of the signal group against Algorithm 4 of
    the oracle applied to the GPU's own triples;
  * k = 130, 200, 255 (d = 260, 400, 510): the cluster kernels with column
    loops over shared memory, the one-CTA projected SVD, and the one-CTA SVD
    without the FP32 preconditioner.
Tolerances: sigma <= 1e-10 relative (F64) / 1e-5 (F32C); reconstructions
<= 1e-9 relative L2 (F64); in F32C the FP32 convolution is held to 1e-5
relative before the division by the antidiagonal counts, and 1e-3 after it
(counts as small as 1 at the ends amplify its error); vectors by the sine of the angle,
allowed 1e-11 sigma_1 / gap by Wedin's bound where the gap is small."""
import os

import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import ssa as ossa
from oracle import trajectory
from paper_0911_4498_gb300 import synth
from ssa_testlib import compare_vectors, gpu_decompose, gpu_decompose_reconstruct

from conftest import GOLDEN, load_golden

pytestmark = pytest.mark.gpu

SIG_F64, SIG_F32C = 1e-10, 1e-5
REC_F64, REC_F32C, CONV_F32C = 1e-9, 1e-3, 1e-5


def _gold(name):
    if not os.path.exists(os.path.join(GOLDEN, name)):
        pytest.skip(f"{name} not generated")
    return load_golden(name)


def _sampled_vectors(g, out, k, n_vec, tol_floor):
    """Entries of u_i, v_i at the stored rows, for the first n_vec triples (sign-aligned)."""
    ref = g["sigma"]
    rows_u = g["rows_u"].astype(np.int64)
    rows_v = g["rows_v"].astype(np.int64)
    for i in range(n_vec):
        gap = min(abs(ref[i] - ref[j]) for j in range(k) if j != i) / ref[0]
        tol = max(tol_floor, 1e-12 / gap)
        su = np.sign(out["U"][rows_u, i] @ g[f"u{i}"])
        assert np.max(np.abs(su * out["U"][rows_u, i] - g[f"u{i}"])) <= tol, i
        assert np.max(np.abs(su * out["V"][rows_v, i] - g[f"v{i}"])) <= tol, i


@pytest.mark.parametrize("precision", [ssa.SSA_PREC_F64, ssa.SSA_PREC_F32C])
def test_standin_N5113_k100_against_golden(precision):
    g = _gold("sigma_three_sines_N5113_L2556_k100.txt")
    N, L, k = int(g["N"][0]), int(g["L"][0]), int(g["k"][0])
    f = synth.three_sines(N, seed=7)
    out = gpu_decompose(f, L, k, precision=precision)
    assert out["rc"] == ssa.SSA_OK and out["info"]["converged"]
    ref = g["sigma"]
    tol = SIG_F64 if precision == ssa.SSA_PREC_F64 else SIG_F32C
    assert np.max(np.abs(out["sigma"] - ref) / ref) <= tol
    if precision != ssa.SSA_PREC_F64:
        return
    _sampled_vectors(g, out, k, 8, 1e-9)
    # relation (1) with the explicit trajectory matrix: X v_i = sigma_i u_i and X^T u_i = sigma_i v_i
    X = trajectory.trajectory_matrix(f, L)
    r1 = np.linalg.norm(X @ out["V"] - out["U"] * out["sigma"], axis=0)
    r2 = np.linalg.norm(X.T @ out["U"] - out["V"] * out["sigma"], axis=0)
    assert max(r1.max(), r2.max()) <= 1e-11 * ref[0]
    # orthonormal returned bases
    for Q in (out["U"], out["V"]):
        assert np.max(np.abs(Q.T @ Q - np.eye(k))) <= 1e-12


@pytest.mark.parametrize("N,L,k", [(1200, 600, 130), (1000, 500, 200), (1100, 550, 255)])
def test_wide_krylov_bases_against_jacobi(N, L, k):
    f = synth.three_sines(N, seed=N + k)
    ref = ossa.decompose(f, L, k, method="jacobi")
    out = gpu_decompose(f, L, k)
    assert out["rc"] == ssa.SSA_OK and out["info"]["converged"]
    assert out["info"]["krylov_dim"] > 256
    assert np.max(np.abs(out["sigma"] - ref["sigma"]) / ref["sigma"]) <= SIG_F64
    nxt = ref["all_sigma"][k]
    compare_vectors(out["U"], ref["U"], ref["sigma"], 1e-9, res_tol=1e-11, sigma_next=nxt)
    compare_vectors(out["V"], ref["V"], ref["sigma"], 1e-9, res_tol=1e-11, sigma_next=nxt)
    X = trajectory.trajectory_matrix(f, L)
    r1 = np.linalg.norm(X @ out["V"] - out["U"] * out["sigma"], axis=0)
    assert r1.max() <= 1e-11 * ref["sigma"][0]


@pytest.fixture(scope="module")
def stress():
    g = _gold("sigma_damped_sines_N4194304_L2097152_k100.txt")
    N, L, k = int(g["N"][0]), int(g["L"][0]), int(g["k"][0])
    return g, synth.damped_sines(N, seed=3), N, L, k


@pytest.mark.parametrize("precision", [ssa.SSA_PREC_F64, ssa.SSA_PREC_F32C])
def test_precision_stress_N4M_against_golden(stress, precision):
    g, f, N, L, k = stress
    signal = 40
    groups = [list(range(signal))]
    out = gpu_decompose_reconstruct(f, L, k, groups, precision=precision)
    assert out["rc"] == ssa.SSA_OK
    ref = g["sigma"]
    d = np.abs(out["sigma"] - ref)
    tol = SIG_F64 if precision == ssa.SSA_PREC_F64 else SIG_F32C
    assert np.max(d[:signal] / ref[:signal]) <= tol          # signal triples, relative
    assert np.max(d / ref[0]) <= tol                         # all 100, against sigma_1 (Weyl)
    if precision == ssa.SSA_PREC_F64:
        _sampled_vectors(g, out, k, 8, 1e-9)
    # reconstruction of the signal group vs Algorithm 4 of the oracle on the same triples
    want = ossa.reconstruct(N, L, out["sigma"], out["U"], out["V"], groups, method="fft", fft="library")
    err = np.linalg.norm(out["rec"][0] - want[0]) / np.linalg.norm(want[0])
    assert err <= (REC_F64 if precision == ssa.SSA_PREC_F64 else REC_F32C), err
    cnt = trajectory.antidiagonal_counts(N, L)
    cerr = np.linalg.norm((out["rec"][0] - want[0]) * cnt) / np.linalg.norm(want[0] * cnt)
    assert cerr <= (REC_F64 if precision == ssa.SSA_PREC_F64 else CONV_F32C), cerr
    # and the signal group is the series without its 1e-6 noise
    assert np.linalg.norm(out["rec"][0] - f) / np.linalg.norm(f) <= 1e-4
