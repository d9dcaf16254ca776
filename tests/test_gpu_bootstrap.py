"""Batched grouped Hankelization and the bootstrap workload of section 6.3:
many noisy replicas of one rank-5 series, each reconstructed from its first
five triples in one batched decomposition + one batched reconstruction."""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import ssa as ossa
from paper_0911_4498_gb300 import synth

pytestmark = pytest.mark.gpu


def _batch(fs, Ls, ks, precision):
    off = np.zeros(len(fs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([f.size for f in fs])
    b, rc = ssa.ssa_decompose_batch(np.concatenate(fs), off, np.asarray(Ls, dtype=np.int64),
                                    np.asarray(ks, dtype=np.int32), ssa.make_opts(precision=precision))
    assert rc == ssa.SSA_OK
    return b


def _recon(b, fs, groups):
    goff, gidx = ssa.groups_csr(groups)
    m = len(groups)
    out = np.empty(sum(m * f.size for f in fs))
    ssa.ssa_batch_reconstruct(b, goff, gidx, m, out)
    res, pos = [], 0
    for f in fs:
        res.append(out[pos:pos + m * f.size].reshape(m, f.size))
        pos += m * f.size
    return res


@pytest.mark.parametrize("precision,tol", [(ssa.SSA_PREC_F64, 1e-9), (ssa.SSA_PREC_F32C, 1e-5)])
def test_batched_reconstruction_matches_oracle(precision, tol):
    # groups follow the sine pairs of the three-sine series (amplitudes 2, 1, 0.5), so
    # each group sum is determined although the triples inside a pair are not
    specs = [(1000, 500, 10), (777, 259, 8), (3001, 1000, 12), (300, 150, 6), (5000, 2500, 8)]
    fs = [synth.three_sines(N, seed=70 + i) for i, (N, _, _) in enumerate(specs)]
    groups = [[0, 1], [2, 3], [4, 5]]
    b = _batch(fs, [s[1] for s in specs], [s[2] for s in specs], precision)
    try:
        got = _recon(b, fs, groups)
    finally:
        ssa.ssa_batch_destroy(b)
    for (N, L, k), f, g in zip(specs, fs, got):
        ref = ossa.decompose(f, L, k, method="jacobi" if N <= 1500 else "lanczos")
        rec = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], groups, method="naive" if N <= 1500 else "fft")
        for gi in range(len(groups)):
            err = np.linalg.norm(g[gi] - rec[gi]) / np.linalg.norm(rec[gi])
            assert err <= tol, (N, L, k, gi, err)


def test_bootstrap_replicas():
    """Rank-5 series: without noise the first five triples give it back exactly;
    with noise (sigma = 5) each replica's rank-5 reconstruction matches the oracle."""
    N, L, R = 1000, 500, 24
    clean = synth.bootstrap_series(N, seed=0, sigma=0.0)
    b = _batch([clean], [L], [5], ssa.SSA_PREC_F64)
    try:
        g = _recon(b, [clean], [list(range(5))])[0][0]
    finally:
        ssa.ssa_batch_destroy(b)
    assert np.linalg.norm(g - clean) <= 1e-9 * np.linalg.norm(clean)

    reps = [synth.bootstrap_series(N, seed=100 + r) for r in range(R)]
    b = _batch(reps, [L] * R, [5] * R, ssa.SSA_PREC_F64)
    try:
        G = np.stack([x[0] for x in _recon(b, reps, [list(range(5))])])
    finally:
        ssa.ssa_batch_destroy(b)
    for r in range(0, R, 6):
        ref = ossa.decompose(reps[r], L, 5, method="jacobi")
        rec = ossa.reconstruct(N, L, ref["sigma"], ref["U"], ref["V"], [list(range(5))], method="naive")[0]
        assert np.linalg.norm(G[r] - rec) <= 1e-9 * np.linalg.norm(rec)
    # the bootstrap statistics: the reconstruction tracks the clean series far better than the noisy input
    mse_rec = np.mean((G - clean) ** 2)
    mse_in = np.mean((np.stack(reps) - clean) ** 2)
    assert mse_rec < 0.1 * mse_in


def test_batched_reconstruction_rejects_bad_groups():
    fs = [synth.three_sines(500, seed=1), synth.three_sines(600, seed=2)]
    b = _batch(fs, [250, 300], [4, 6], ssa.SSA_PREC_F64)
    try:
        out = np.empty(2 * 1100)
        for groups in ([[0, 4]], [[0, 1], [1]]):           # index >= min k; overlap
            off, idx = ssa.groups_csr(groups)
            with pytest.raises(ssa.SSAError):
                ssa.ssa_batch_reconstruct(b, off, idx, len(groups), out)
    finally:
        ssa.ssa_batch_destroy(b)
