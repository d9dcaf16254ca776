"""Request server (continuous batching): results of a mixed stream of
requests match the oracle, each result is the same alone and in the mix,
admission respects the memory budget, and running requests overlap.  In
FP32-compensated mode vectors are compared for triples with sigma_i >=
1e-2 sigma_1: below that the FP32 product error (~1e-7 sigma_1) exceeds the
gaps of the noise bulk, so those vectors are not determined to 1e-4."""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import ssa as ossa
from paper_0911_4498_gb300 import synth
from ssa_testlib import compare_vectors

pytestmark = pytest.mark.gpu

# (N, L, k): batched (small N, k <= 36) and single-series requests, ragged
MIX = [(1000, 500, 10), (777, 259, 4), (5000, 2500, 16), (20000, 6667, 12), (3000, 1500, 40),
       (40000, 20000, 8), (1500, 750, 30), (120000, 60000, 20), (64, 32, 5), (9000, 3000, 24)]
SIG_F32C = 1e-5


def _series(i, N):
    return synth.three_sines(N, seed=5000 + i)


def _serve(specs, opts=None, outputs=ssa.SSA_SERVE_VECTORS, stagger=0.0):
    import time
    srv = ssa.ssa_serve_create(opts if opts is not None else ssa.make_serve_opts())
    try:
        ids = []
        for i, (N, L, k) in enumerate(specs):
            ids.append(ssa.ssa_serve_submit(srv, _series(i, N), L, k, outputs))
            if stagger:
                time.sleep(stagger)
        out = []
        for rid, (N, L, k) in zip(ids, specs):
            while not ssa.ssa_serve_poll(srv, rid, 5.0):
                pass
            sig = np.empty(k)
            U = np.empty((k, L)) if outputs else None
            V = np.empty((k, N - L + 1)) if outputs else None
            rc, info = ssa.ssa_serve_take(srv, rid, sig, U, V, None)
            out.append({"sigma": sig, "U": None if U is None else U.T.copy(), "V": None if V is None else V.T.copy(),
                        "info": info, "rc": rc})
        stats = ssa.ssa_serve_stats(srv)
    finally:
        ssa.ssa_serve_destroy(srv)
    return out, stats


def test_mixed_stream_matches_oracle():
    out, stats = _serve(MIX)
    assert stats["completed"] == len(MIX) and stats["queued"] == 0 and stats["running"] == 0
    assert stats["batches"] >= 1 and 0 < stats["batched_requests"] < len(MIX)
    for i, ((N, L, k), o) in enumerate(zip(MIX, out)):
        assert o["rc"] == ssa.SSA_OK and o["info"]["converged"]
        ref = ossa.decompose(_series(i, N), L, k, method="jacobi" if N <= 1500 else "lanczos")
        rel = np.max(np.abs(o["sigma"] - ref["sigma"]) / ref["sigma"])
        assert rel <= SIG_F32C, (N, L, k, rel)
        # FP32 products: residuals up to ~1e-6 sigma_1, vectors within Wedin's bound
        compare_vectors(o["U"], ref["U"], ref["sigma"], 1e-4, skip_below=1e-2 * ref["sigma"][0], res_tol=1e-6)


def test_each_result_same_alone_and_in_the_mix():
    mix, _ = _serve(MIX, stagger=0.002)
    for j in range(len(MIX)):
        N, L, k = MIX[j]
        srv = ssa.ssa_serve_create(ssa.make_serve_opts())
        try:
            rid = ssa.ssa_serve_submit(srv, _series(j, N), L, k, ssa.SSA_SERVE_VECTORS)
            while not ssa.ssa_serve_poll(srv, rid, 5.0):
                pass
            sig = np.empty(k)
            U = np.empty((k, L))
            rc, info = ssa.ssa_serve_take(srv, rid, sig, U, None, None)
        finally:
            ssa.ssa_serve_destroy(srv)
        assert rc == ssa.SSA_OK
        assert info["batched"] == mix[j]["info"]["batched"]
        rel = np.max(np.abs(sig - mix[j]["sigma"]) / mix[j]["sigma"])
        assert rel <= 1e-6, (MIX[j], rel)
        compare_vectors(U.T.copy(), mix[j]["U"], sig, 1e-5, skip_below=1e-2 * sig[0], res_tol=1e-6)


@pytest.mark.parametrize("grid_cap", [0, 24])
def test_f64_server_matches_plan_path(grid_cap):
    """FP64 requests through the server (whole-device grids, or capped to 24 CTAs per persistent
    kernel) give the plan path's sigma to the FP64 tolerance; a negative cap is refused."""
    from ssa_testlib import gpu_decompose
    specs = [(1000, 500, 10), (30000, 15000, 12), (2000, 1000, 40), (70000, 35000, 8)]
    out, _ = _serve(specs, ssa.make_serve_opts(precision=ssa.SSA_PREC_F64, grid_cap=grid_cap))
    for i, ((N, L, k), o) in enumerate(zip(specs, out)):
        p = gpu_decompose(_series(i, N), L, k)
        assert np.max(np.abs(p["sigma"] - o["sigma"]) / p["sigma"]) <= 1e-10
    with pytest.raises(ssa.SSAError):
        ssa.ssa_serve_create(ssa.make_serve_opts(grid_cap=-1))


def test_budget_admission_and_overlap():
    specs = [(60000, 30000, 16)] * 6 + [(2000, 1000, 8)] * 20
    # a budget for about two of the single-series requests (~60 MB each) at a time
    budget = 128 << 20
    out, stats = _serve(specs, ssa.make_serve_opts(mem_budget=budget, workers=8), outputs=0)
    assert all(o["rc"] == ssa.SSA_OK for o in out)
    assert stats["mem_peak"] <= budget
    out2, stats2 = _serve(specs, ssa.make_serve_opts(workers=8), outputs=0)
    # with the default budget several single-series requests run at once
    single = [o["info"] for o in out2 if not o["info"]["batched"]]
    overlaps = sum(1 for a in single for b in single if a is not b and a["t_start"] < b["t_done"] and b["t_start"] < a["t_done"])
    assert overlaps > 0
    assert stats2["mem_peak"] > stats["mem_peak"]


def test_sigma_only_outputs_and_errors():
    srv = ssa.ssa_serve_create(ssa.make_serve_opts(mem_budget=1 << 26))
    try:
        f = _series(0, 1000)
        with pytest.raises(ssa.SSAError):
            ssa.ssa_serve_submit(srv, f, 1000, 3)          # L >= N
        with pytest.raises(ssa.SSAError):
            ssa.ssa_serve_submit(srv, f, 500, 0)           # k < 1
        with pytest.raises(ssa.SSAError):                  # beyond the 64 MiB budget
            ssa.ssa_serve_submit(srv, _series(1, 1 << 20), 1 << 19, 50)
        rid = ssa.ssa_serve_submit(srv, f, 500, 10)
        while not ssa.ssa_serve_poll(srv, rid, 5.0):
            pass
        with pytest.raises(ssa.SSAError):                  # vectors were not requested
            ssa.ssa_serve_take(srv, rid, np.empty(10), np.empty((10, 500)), None, None)
        sig = np.empty(10)
        rc, info = ssa.ssa_serve_take(srv, rid, sig)
        assert rc == ssa.SSA_OK and info["batched"] == 1 and sig[0] > sig[-1] > 0
        with pytest.raises(ssa.SSAError):                  # already released
            ssa.ssa_serve_take(srv, rid, np.empty(10))
    finally:
        ssa.ssa_serve_destroy(srv)
