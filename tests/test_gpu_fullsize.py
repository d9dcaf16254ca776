"""Full-size parity at the benchmark workload (N = 2^20, L = 2^19, k = 50) in the
launch configuration bench.py times: singular values against the oracle's stored
values (tests/golden, written by make_golden.py from the oracle only), sampled
vector entries, and relation A v_i = sigma_i u_i checked row by row from the
definition X[i, :] . v = sum_m f[i+m] v[m]."""
import os

import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from paper_0911_4498_gb300 import synth
from ssa_testlib import gpu_decompose_reconstruct

from conftest import load_golden

pytestmark = pytest.mark.gpu

GOLD = "sigma_many_sines_N1048576_L524288_k50.txt"


def _gold():
    if not os.path.exists(os.path.join(os.path.dirname(__file__), "golden", GOLD)):
        pytest.skip("golden values not generated")
    return load_golden(GOLD)


def _run(precision):
    g = _gold()
    N, L, k = int(g["N"][0]), int(g["L"][0]), int(g["k"][0])
    f = synth.many_sines(N, seed=1)
    groups = [[0, 1], [2], [3]]
    out = gpu_decompose_reconstruct(f, L, k, groups, precision=precision)
    return g, f, N, L, k, out


def test_fullsize_f64_sigma_vectors_relation():
    g, f, N, L, k, out = _run(ssa.SSA_PREC_F64)
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
    # grouped reconstruction is finite and Hankel-consistent with the vectors
    assert np.all(np.isfinite(out["rec"]))


def test_fullsize_f32c_sigma():
    g, f, N, L, k, out = _run(ssa.SSA_PREC_F32C)
    ref = g["sigma"]
    rel = np.abs(out["sigma"] - ref) / ref
    assert np.max(rel) <= 1e-5, rel
