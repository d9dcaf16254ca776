"""Batched decompositions (one persistent launch over ragged series): each series
matches the oracle, and each result is the same alone and in the mix."""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import ssa as ossa
from paper_0911_4498_gb300 import synth
from ssa_testlib import compare_vectors

pytestmark = pytest.mark.gpu

MIX = [(37, 12, 3), (500, 250, 8), (1000, 500, 10), (777, 259, 12), (2049, 683, 6), (5000, 2500, 16),
       (120, 90, 5), (3000, 1000, 32), (64, 32, 20), (1500, 750, 4), (9000, 4500, 10), (20000, 6667, 12)]


def _run_batch(specs, precision, seed=0):
    fs = [synth.three_sines(N, seed=1000 + i) for i, (N, L, k) in enumerate(specs)]
    off = np.zeros(len(specs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([f.size for f in fs])
    f_all = np.concatenate(fs)
    Ls = np.array([L for _, L, _ in specs], dtype=np.int64)
    ks = np.array([k for _, _, k in specs], dtype=np.int32)
    b, rc = ssa.ssa_decompose_batch(f_all, off, Ls, ks, ssa.make_opts(precision=precision, seed=seed))
    out = []
    try:
        for i, (N, L, k) in enumerate(specs):
            K = N - L + 1
            sig = np.empty(k)
            U = np.empty((k, L))
            V = np.empty((k, K))
            ssa.ssa_batch_get(b, i, sig, U, V, None)
            out.append({"f": fs[i], "sigma": sig, "U": U.T.copy(), "V": V.T.copy(), "info": ssa.ssa_batch_info(b, i)})
    finally:
        ssa.ssa_batch_destroy(b)
    return out, rc


@pytest.mark.parametrize("precision", [ssa.SSA_PREC_F32C, ssa.SSA_PREC_F64])
def test_batch_matches_oracle(precision):
    specs = MIX if precision == ssa.SSA_PREC_F32C else [s for s in MIX if s[0] <= 16384]
    out, rc = _run_batch(specs, precision)
    assert rc == ssa.SSA_OK
    tol = 1e-5 if precision == ssa.SSA_PREC_F32C else 1e-10
    for (N, L, k), o in zip(specs, out):
        ref = ossa.decompose(o["f"], L, k, method="jacobi" if N <= 1500 else "lanczos")
        rel = np.max(np.abs(o["sigma"] - ref["sigma"]) / ref["sigma"])
        assert rel <= tol, (N, L, k, rel)
        assert o["info"]["converged"]
        if precision == ssa.SSA_PREC_F64:
            compare_vectors(o["U"], ref["U"], ref["sigma"], 1e-7)
            compare_vectors(o["V"], ref["V"], ref["sigma"], 1e-7)


@pytest.mark.parametrize("precision,tol", [(ssa.SSA_PREC_F32C, 1e-6), (ssa.SSA_PREC_F64, 1e-10)])
def test_each_result_same_alone_and_in_the_mix(precision, tol):
    specs = MIX if precision == ssa.SSA_PREC_F32C else [s for s in MIX if s[0] <= 16384]
    mix, _ = _run_batch(specs, precision)
    for j in [0, 5, len(specs) - 1]:
        N, L, k = specs[j]
        fj = synth.three_sines(N, seed=1000 + j)
        off = np.array([0, N], dtype=np.int64)
        b, rc = ssa.ssa_decompose_batch(fj, off, np.array([L], dtype=np.int64), np.array([k], dtype=np.int32),
                                        ssa.make_opts(precision=precision))
        try:
            assert rc == ssa.SSA_OK
            sig = np.empty(k)
            U = np.empty((k, L))
            ssa.ssa_batch_get(b, 0, sig, U, None, None)
        finally:
            ssa.ssa_batch_destroy(b)
        rel = np.max(np.abs(sig - mix[j]["sigma"]) / mix[j]["sigma"])
        assert rel <= tol, (specs[j], rel)
        # FP32 products: Ritz residuals up to ~1e-6 sigma_1 (Wedin bound); df64: rounding only
        if precision == ssa.SSA_PREC_F32C:
            compare_vectors(U.T.copy(), mix[j]["U"], sig, 1e-5, res_tol=1e-6)
        else:
            compare_vectors(U.T.copy(), mix[j]["U"], sig, 1e-7)


def test_batch_agrees_with_plan_path():
    specs = [(1000, 500, 10), (5000, 2500, 16)]
    out, _ = _run_batch(specs, ssa.SSA_PREC_F64)
    from ssa_testlib import gpu_decompose
    for (N, L, k), o in zip(specs, out):
        p = gpu_decompose(o["f"], L, k)
        assert np.max(np.abs(p["sigma"] - o["sigma"]) / p["sigma"]) <= 1e-10


def test_batch_rejects_bad_sizes():
    f = synth.three_sines(100, 1)
    with pytest.raises(ssa.SSAError):
        ssa.ssa_decompose_batch(f, np.array([0, 100], dtype=np.int64), np.array([100], dtype=np.int64),
                                np.array([3], dtype=np.int32))
    f = synth.three_sines(1000, 1)
    one = np.array([0, 1000], dtype=np.int64)
    with pytest.raises(ssa.SSAError):   # k = 45 needs a Krylov dimension of 90, beyond the batched limit 72
        ssa.ssa_decompose_batch(f, one, np.array([500], dtype=np.int64), np.array([45], dtype=np.int32))
    f = synth.three_sines(20000, 1)
    with pytest.raises(ssa.SSAError):   # refinement in a batch needs N <= 16384
        ssa.ssa_decompose_batch(f, np.array([0, 20000], dtype=np.int64), np.array([6667], dtype=np.int64),
                                np.array([8], dtype=np.int32),
                                ssa.make_opts(precision=ssa.SSA_PREC_F32C, refine=ssa.SSA_REFINE_ON))


def _rayleigh(f, L, U, V):
    """u_i^T X v_i with the oracle's FP64 products."""
    from oracle import fast_hankel
    chat = fast_hankel.spectrum(f, L, fast_hankel.fft_length(f.size))
    XV = np.stack([fast_hankel.hankel_matvec(chat, f.size, L, V[:, i]) for i in range(V.shape[1])], axis=1)
    return np.einsum("ij,ij->j", U, XV)


@pytest.mark.parametrize("precision", [ssa.SSA_PREC_F32C, ssa.SSA_PREC_F64])
def test_batch_refinement_is_the_rayleigh_quotient(precision):
    """With refinement each returned sigma_i is u_i^T X v_i of the returned
    vectors (FP64), sorted, and still within the precision's tolerance."""
    specs = [s for s in MIX if s[0] <= 16384]
    fs = [synth.three_sines(N, seed=1000 + i) for i, (N, L, k) in enumerate(specs)]
    off = np.zeros(len(specs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([f.size for f in fs])
    b, rc = ssa.ssa_decompose_batch(np.concatenate(fs), off, np.array([L for _, L, _ in specs], dtype=np.int64),
                                    np.array([k for _, _, k in specs], dtype=np.int32),
                                    ssa.make_opts(precision=precision, refine=ssa.SSA_REFINE_ON))
    tol = 1e-5 if precision == ssa.SSA_PREC_F32C else 1e-10
    try:
        assert rc == ssa.SSA_OK
        for i, (N, L, k) in enumerate(specs):
            K = N - L + 1
            sig = np.empty(k)
            U = np.empty((k, L))
            V = np.empty((k, K))
            ssa.ssa_batch_get(b, i, sig, U, V, None)
            rq = _rayleigh(fs[i], L, U.T.copy(), V.T.copy())
            assert np.max(np.abs(sig - rq)) <= 1e-12 * sig[0], (N, L, k)
            assert np.all(np.diff(sig) <= 0)
            ref = ossa.decompose(fs[i], L, k, method="jacobi" if N <= 1500 else "lanczos")
            assert np.max(np.abs(sig - ref["sigma"]) / ref["sigma"]) <= tol, (N, L, k)
            assert ssa.ssa_batch_info(b, i)["matvecs"] > 0
    finally:
        ssa.ssa_batch_destroy(b)


@pytest.mark.slow
def test_full_size_batch_sampled():
    """The 4096-series batch exactly as bench.py times it (F32C, one launch):
    every series converges with sorted sigma, and sampled series match the oracle."""
    fs, Ls, ks = synth.batch_workload(4096, seed=2)
    off = np.zeros(len(fs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([f.size for f in fs])
    b, rc = ssa.ssa_decompose_batch(np.concatenate(fs), off, Ls.astype(np.int64), ks.astype(np.int32),
                                    ssa.make_opts(precision=ssa.SSA_PREC_F32C))
    try:
        assert rc == ssa.SSA_OK
        for i in range(len(fs)):
            assert ssa.ssa_batch_info(b, i)["converged"]
        for i in [0, 1, 777, 2048, 4095]:
            sig = np.empty(int(ks[i]))
            ssa.ssa_batch_get(b, i, sig, None, None, None)
            assert np.all(np.diff(sig) <= 0)
            ref = ossa.decompose(fs[i], int(Ls[i]), int(ks[i]), method="lanczos")
            assert np.max(np.abs(sig - ref["sigma"]) / ref["sigma"]) <= 1e-5, i
    finally:
        ssa.ssa_batch_destroy(b)


def test_plan_run_wait_and_cuda_graph_replay():
    """ssa_batch_plan / ssa_batch_run / ssa_batch_wait give the results of
    ssa_decompose_batch, and a run captured in a CUDA graph replays on new
    series data in the same buffer."""
    import torch
    specs = [s for s in MIX if s[0] <= 16384]
    Ns = [N for N, _, _ in specs]
    off = np.zeros(len(specs) + 1, dtype=np.int64)
    off[1:] = np.cumsum(Ns)
    Ls = np.array([L for _, L, _ in specs], dtype=np.int64)
    ks = np.array([k for _, _, k in specs], dtype=np.int32)
    fa = np.concatenate([synth.three_sines(N, seed=300 + i) for i, N in enumerate(Ns)])
    fb = np.concatenate([synth.three_sines(N, seed=400 + i) for i, N in enumerate(Ns)])

    def direct(f):
        b, rc = ssa.ssa_decompose_batch(f, off, Ls, ks, ssa.make_opts(precision=ssa.SSA_PREC_F32C))
        try:
            return [_sig(b, i, k) for i, k in enumerate(ks)]
        finally:
            ssa.ssa_batch_destroy(b)

    side = torch.cuda.Stream()
    plan = ssa.ssa_batch_plan(off, Ls, ks, ssa.make_opts(precision=ssa.SSA_PREC_F32C, stream=side.cuda_stream))
    try:
        fd = torch.from_numpy(fa).cuda()
        torch.cuda.synchronize()
        ssa.ssa_batch_run(plan, fd)
        assert ssa.ssa_batch_wait(plan) == ssa.SSA_OK
        for got, ref in zip([_sig(plan, i, k) for i, k in enumerate(ks)], direct(fa)):
            np.testing.assert_array_equal(got, ref)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            ssa.ssa_batch_run(plan, fd)
        fd.copy_(torch.from_numpy(fb))
        torch.cuda.synchronize()
        g.replay()                 # launches on the current stream, not on the plan's stream
        torch.cuda.synchronize()
        assert ssa.ssa_batch_wait(plan) == ssa.SSA_OK
        for got, ref in zip([_sig(plan, i, k) for i, k in enumerate(ks)], direct(fb)):
            np.testing.assert_array_equal(got, ref)
    finally:
        ssa.ssa_batch_destroy(plan)


def _sig(b, i, k):
    out = np.empty(int(k))
    ssa.ssa_batch_get(b, i, out, None, None, None)
    return out
