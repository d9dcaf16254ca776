"""Error paths of the single-series calls, made to happen on the host:

  * SSA_ENOCONV: with max_restarts = 0 the first Krylov cycle is all there
    is; the call still returns sigma, vectors and residuals, the residuals
    show what did not converge, and the result can be reconstructed;
  * SSA_ENOMEM: ssa_fault_inject_alloc makes the n-th device allocation fail
    (no allocator is called, nothing fails on the device) for every n the
    plan, decomposition and reconstruction make; each call returns
    SSA_ENOMEM, and afterwards the library gives the oracle's result again.
"""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from oracle import ssa as ossa
from paper_0911_4498_gb300 import synth

pytestmark = pytest.mark.gpu


def test_no_convergence_returns_results_and_residuals():
    N, L, k = 5000, 2500, 10
    f = synth.many_sines(N, seed=5)
    ref = ossa.decompose(f, L, k, method="lanczos")
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(max_restarts=0, krylov_dim=k + 4))
    try:
        d, rc = ssa.ssa_decompose(plan, f, k)
        try:
            assert rc == ssa.SSA_ENOCONV
            info = ssa.ssa_decomp_info(d)
            assert not info["converged"] and info["restarts"] == 0
            sigma, resid = np.empty(k), np.empty(k)
            U, V = np.empty((k, L)), np.empty((k, N - L + 1))
            ssa.ssa_decomp_get(d, sigma, U, V, resid)
            assert np.all(np.isfinite(sigma)) and np.all(np.isfinite(resid))
            assert np.all(np.diff(sigma) <= 0)
            # Ritz values of one cycle are below the true ones (interlacing) and not converged
            assert np.all(sigma <= ref["sigma"] * (1 + 1e-12))
            assert np.max(resid) > 1e-12 * sigma[0]
            # relation (2): the residual bounds each Ritz value's distance to a singular value
            # (up to the products' rounding, ~1e-14 sigma_1)
            for i in range(k):
                assert np.min(np.abs(ref["sigma"] - sigma[i])) <= resid[i] * (1 + 1e-6) + 1e-12 * sigma[0] or \
                    sigma[i] < ref["sigma"][-1]
            off, idx = ssa.groups_csr([[0, 1]])
            out = np.empty((1, N))
            ssa.ssa_reconstruct(d, off, idx, 1, out)
            assert np.all(np.isfinite(out))
        finally:
            ssa.ssa_decomp_destroy(d)
    finally:
        ssa.ssa_plan_destroy(plan)


def _run(f, L, k):
    """Plan, decompose, reconstruct; returns the first failing status or the sigma."""
    N = f.size
    try:
        plan = ssa.ssa_embed_plan(N, L, ssa.make_opts())
    except ssa.SSAError as e:
        return e.code
    try:
        try:
            d, rc = ssa.ssa_decompose(plan, f, k)
        except ssa.SSAError as e:
            return e.code
        try:
            sigma = np.empty(k)
            ssa.ssa_decomp_get(d, sigma, None, None, None)
            off, idx = ssa.groups_csr([[0], [1, 2]])
            out = np.empty((2, N))
            try:
                ssa.ssa_reconstruct(d, off, idx, 2, out)
            except ssa.SSAError as e:
                return e.code
            return sigma
        finally:
            ssa.ssa_decomp_destroy(d)
    finally:
        ssa.ssa_plan_destroy(plan)


@pytest.mark.parametrize("N,L", [(1000, 500), (40000, 13000)])
def test_injected_allocation_failures(N, L):
    k = 6
    f = synth.three_sines(N, seed=9)
    ref = ossa.decompose(f, L, k, method="jacobi" if N <= 1500 else "lanczos")
    failures = 0
    try:
        for after in range(200):
            ssa.ssa_fault_inject_alloc(after)
            r = _run(f, L, k)
            if isinstance(r, int):
                assert r == ssa.SSA_ENOMEM, (after, r)
                failures += 1
                continue
            # the injection point lies beyond the last allocation: a normal result
            assert np.max(np.abs(r - ref["sigma"]) / ref["sigma"]) <= 1e-10
            break
        else:
            pytest.fail("the calls made more than 200 allocations")
    finally:
        ssa.ssa_fault_inject_alloc(-1)
    assert failures >= 10
    # the library works normally afterwards
    r = _run(f, L, k)
    assert not isinstance(r, int)
    assert np.max(np.abs(r - ref["sigma"]) / ref["sigma"]) <= 1e-10
