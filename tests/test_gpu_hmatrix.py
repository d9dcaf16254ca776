"""H-matrix (section 6.4) on the GPU against the oracle's definition."""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import hmatrix as ohm
from paper_0911_4498_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def paper_case():
    # the section 6.4 example: N = 400, Q = 200, B = T = 100, L = 50, I = {1, 2}
    f = synth.hmatrix_series(400, 200, seed=0)
    return f, ohm.hmatrix(f, 50, 100, 100, [1, 2])


@pytest.mark.parametrize("precision,tol", [(ssa.SSA_PREC_F64, 1e-9), (ssa.SSA_PREC_F32C, 1e-5)])
def test_paper_example_matches_oracle(paper_case, precision, tol):
    f, ref = paper_case
    G, rc = ssa.ssa_hmatrix(f, 50, 100, 100, [1, 2], ssa.make_opts(precision=precision))
    assert rc == ssa.SSA_OK
    assert G.shape == ref.shape == (301, 301)
    assert np.max(np.abs(G - ref)) <= tol
    # the structure the paper shows: homogeneous blocks near 0, cross blocks clearly above
    assert np.max(G[:50, :50]) < 0.01 and np.min(G[:50, -50:]) > 0.05


def test_plan_path_per_window_and_device_buffers():
    """k beyond the batched engine's Krylov limit: one plan per base window."""
    import torch
    f = synth.hmatrix_series(300, 150, seed=2)
    L, B, T, I = 60, 120, 80, [1, 2, 40]
    ref = ohm.hmatrix(f, L, B, T, I)
    fd = torch.from_numpy(f).cuda()
    out = torch.empty((300 - B + 1, 300 - T + 1), dtype=torch.float64, device="cuda")
    _, rc = ssa.ssa_hmatrix(fd, L, B, T, I, ssa.make_opts(), out=out)
    assert rc == ssa.SSA_OK
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-9


def test_ragged_sizes():
    f = synth.three_sines(500, seed=9)
    for (L, B, T, I) in [(33, 100, 33, [1]), (40, 257, 301, [2, 3]), (100, 500, 150, [1, 2, 3])]:
        ref = ohm.hmatrix(f, L, B, T, I)
        G, _ = ssa.ssa_hmatrix(f, L, B, T, I)
        assert np.max(np.abs(G - ref)) <= 1e-9, (L, B, T, I)


def test_rejects_bad_parameters():
    f = synth.hmatrix_series(200, 100, seed=1)
    for args in [(50, 50, 60, [1]), (50, 100, 40, [1]), (50, 100, 60, [0]), (50, 100, 60, [1, 1]),
                 (50, 100, 60, [52]), (50, 201, 60, [1])]:
        with pytest.raises(ssa.SSAError):
            ssa.ssa_hmatrix(f, *args)


@pytest.mark.slow
def test_full_size_sampled_rows():
    """The section 6.4 timing setup as bench.py runs it (N = 4000, Q = N/2,
    B = T = N/4, L = B/2, I = {1, 2}): sampled rows against the definition."""
    from oracle import trajectory
    N = 4000
    B = T = N // 4
    L = B // 2
    f = synth.hmatrix_series(N, N // 2, seed=0)
    G, rc = ssa.ssa_hmatrix(f, L, B, T, [1, 2])
    assert rc == ssa.SSA_OK and G.shape == (N - B + 1, N - T + 1)
    assert np.all(G >= 0) and np.all(G <= 1)
    for i in (0, 1500, N - B):
        U = ohm.base_vectors(f[i:i + B], L, [1, 2])
        for j in range(0, N - T + 1, 211):
            X = trajectory.trajectory_matrix(f[j:j + T], L)
            R = X - U @ (U.T @ X)
            assert abs(G[i, j] - np.sum(R * R) / np.sum(X * X)) <= 1e-9, (i, j)
