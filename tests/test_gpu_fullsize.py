"""Full-size parity at the benchmark workload (N = 2^20, L = 2^19, k = 50) in the
launch configuration bench.py times: singular values against the oracle's stored
values (tests/golden, written by make_golden.py from the oracle only), sampled
vector entries, relation A v_i = sigma_i u_i checked row by row from the
definition X[i, :] . v = sum_m f[i+m] v[m], and all 50 elementary
reconstructions element by element against Algorithm 4 of the oracle applied
to the GPU's own triples (numpy's FFT, pinned to the oracle's radix-2 FFT)."""
import os

import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from paper_0911_4498_gb300 import synth
from oracle import ssa as ossa
from ssa_testlib import gpu_decompose_reconstruct

from conftest import load_golden

pytestmark = pytest.mark.gpu

GOLD = "sigma_many_sines_N1048576_L524288_k50.txt"


def _gold():
    if not os.path.exists(os.path.join(os.path.dirname(__file__), "golden", GOLD)):
        pytest.skip("golden values not generated")
    return load_golden(GOLD)


def _run(precision, k=None, **kw):
    g = _gold()
    N, L = int(g["N"][0]), int(g["L"][0])
    k = int(g["k"][0]) if k is None else k
    f = synth.many_sines(N, seed=1)
    groups = [[i] for i in range(k)]       # the bench reconstructs every elementary component
    out = gpu_decompose_reconstruct(f, L, k, groups, precision=precision, **kw)
    return g, f, N, L, k, out


def _check_reconstruction(out, N, L, k, tol, conv_tol=None):
    """Elementary reconstructions vs Algorithm 4 of the oracle on the same triples: relative L2
    error <= tol; with conv_tol also the error of the convolution itself (before the division
    by the antidiagonal counts, which amplifies an FFT's uniform error by up to L/count near
    the ends of the series) relative to the convolution, <= conv_tol."""
    from oracle import trajectory
    groups = [[i] for i in range(k)]
    want = ossa.reconstruct(N, L, out["sigma"], out["U"], out["V"], groups, method="fft", fft="library")
    err = np.linalg.norm(out["rec"] - want, axis=1) / np.linalg.norm(want, axis=1)
    assert np.all(err <= tol), (int(np.argmax(err / tol)), float(np.max(err / tol)))
    if conv_tol is not None:
        cnt = trajectory.antidiagonal_counts(N, L)
        cerr = np.linalg.norm((out["rec"] - want) * cnt, axis=1) / np.linalg.norm(want * cnt, axis=1)
        assert np.max(cerr) <= conv_tol, (int(np.argmax(cerr)), float(np.max(cerr)))
    # the components add up to the series up to the discarded tail (sigma_51.. of a noisy series)
    assert np.linalg.norm(out["rec"].sum(axis=0) - want.sum(axis=0)) <= np.min(tol) * np.linalg.norm(want.sum(axis=0))


# partial reorthogonalisation keeps the bases orthogonal to sqrt(eps) of the double-float products
# (eps = 2^-46); the coefficients it leaves out of B are of that size, so the singular values stay
# at full accuracy (their error is second order) while the vectors and the reconstructions are held
# to sqrt(eps), or to Wedin's bound with a residual of 1e-9 sigma_1 where a gap is small
SQRT_EPS = 2.0 ** -23
PRO_RES = 1e-9


@pytest.mark.parametrize("reorth_skip", [0.0, 1e-12])
def test_fullsize_f64_sigma_vectors_relation(reorth_skip):
    """Both reorthogonalisation settings with FP64-class vectors: full Gram-Schmidt (default) and
    the skip test at 1e-12."""
    g, f, N, L, k, out = _run(ssa.SSA_PREC_F64, reorth_skip=reorth_skip)
    K = N - L + 1
    assert out["rc"] == ssa.SSA_OK
    ref = g["sigma"]
    rel = np.abs(out["sigma"] - ref) / ref
    assert np.max(rel) <= 1e-10, rel
    # sampled entries of the leading well-separated vectors (sign rule on both sides)
    rows_u = g["rows_u"].astype(np.int64)
    rows_v = g["rows_v"].astype(np.int64)
    for i in range(8):
        gap = min(abs(ref[i] - ref[j]) for j in range(k) if j != i) / ref[0]
        tol = max(1e-9, 1e-13 / gap)
        su = np.sign(out["U"][rows_u, i] @ g[f"u{i}"])
        assert np.max(np.abs(su * out["U"][rows_u, i] - g[f"u{i}"])) <= tol * 10
        assert np.max(np.abs(su * out["V"][rows_v, i] - g[f"v{i}"])) <= tol * 10
    # relation (1): X v_i = sigma_i u_i on sampled rows, from the definition
    for i in [0, 5, 20, 49]:
        for row in [0, 1, 4321, L // 2, L - 1]:
            lhs = f[row:row + K] @ out["V"][:, i]
            assert abs(lhs - out["sigma"][i] * out["U"][row, i]) <= 1e-11 * ref[0]
    # every elementary reconstruction, element by element (Algorithm 4, section 5)
    _check_reconstruction(out, N, L, k, 1e-9)


PRO_K = 12   # one Lanczos cycle (the default Krylov dimension 44) converges for these triples


def test_fullsize_f64_partial_reorthogonalisation():
    """PRO at the benchmark's series and window for the 12 leading triples (one cycle, no restart):
    sigma against the stored oracle values at the FP64 tolerance, vectors, relation (1) and the
    12 elementary reconstructions at the semi-orthogonality level."""
    g, f, N, L, k, out = _run(ssa.SSA_PREC_F64, k=PRO_K, reorth=ssa.SSA_REORTH_PRO)
    K = N - L + 1
    assert out["rc"] == ssa.SSA_OK and out["info"]["restarts"] == 0
    ref = g["sigma"][:k]
    assert np.max(np.abs(out["sigma"] - ref) / ref) <= 1e-10
    allsig = g["sigma"]    # gaps also to the first singular values not requested
    gaps = np.array([min(abs(allsig[i] - allsig[j]) for j in range(allsig.size) if j != i)
                     for i in range(k)]) / ref[0]
    rows_u = g["rows_u"].astype(np.int64)
    rows_v = g["rows_v"].astype(np.int64)
    for i in range(8):
        tol = max(SQRT_EPS, PRO_RES / gaps[i])
        su = np.sign(out["U"][rows_u, i] @ g[f"u{i}"])
        assert np.max(np.abs(su * out["U"][rows_u, i] - g[f"u{i}"])) <= tol, i
        assert np.max(np.abs(su * out["V"][rows_v, i] - g[f"v{i}"])) <= tol, i
    for i in [0, 5, k - 1]:
        for row in [0, 1, 4321, L // 2, L - 1]:
            lhs = f[row:row + K] @ out["V"][:, i]
            assert abs(lhs - out["sigma"][i] * out["U"][row, i]) <= PRO_RES * ref[0]
    _check_reconstruction(out, N, L, k, np.maximum(10 * SQRT_EPS, 2 * PRO_RES / gaps))


def test_fullsize_f32c_sigma():
    g, f, N, L, k, out = _run(ssa.SSA_PREC_F32C)
    ref = g["sigma"]
    rel = np.abs(out["sigma"] - ref) / ref
    assert np.max(rel) <= 1e-5, rel
    # FP32 convolutions: ~1e-6 relative; divided by counts as small as 1 at the ends (L = 2^19)
    _check_reconstruction(out, N, L, k, 1e-3, conv_tol=1e-5)
