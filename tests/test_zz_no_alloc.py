"""ssa_matvec_noalloc: the product entry point that allocates no device memory
(its scratch is a fixed file-scope device array) must give the same result as
the plan-based ssa_matvec, call after call.

This file is collected last so that, in a run that stops at the first failure,
every other test has already run.  It passes alone in a fresh process and after
the rest of the suite, since the shared scratch array carries nothing over
between calls that the next call relies on.
"""
import numpy as np
import pytest

import paper_0911_4498_gb300 as ssa
from paper_0911_4498_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-13   # normwise, the double-float product tolerance of the spectral tests
TOL_F32C = 3e-6


def _plan_product(f, L, x, transpose, precision):
    N = f.size
    K = N - L + 1
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=precision))
    try:
        ssa.ssa_set_series(plan, f)
        y = np.empty(K if transpose else L)
        ssa.ssa_matvec(plan, transpose, np.ascontiguousarray(x), y, 1)
        return y
    finally:
        ssa.ssa_plan_destroy(plan)


def _noalloc_product(f, L, x, transpose, precision):
    import torch
    N = f.size
    K = N - L + 1
    fd = torch.from_numpy(f).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.empty(K if transpose else L, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ssa.ssa_matvec_noalloc(fd, N, L, transpose, xd, yd, precision, stream.cuda_stream)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


# (30000, *): n = 16384, the largest single-CTA FP32 product, whose direct
# twiddle table fills its slot of the array exactly; its df64 spectrum takes
# the four-step kernels with that table
CASES = [(1000, 500, 0), (40000, 13000, 1), (65536, 32768, 0), (777, 600, 1), (65536, 50000, 1),
         (30000, 15000, 0), (30000, 20000, 1)]


@pytest.mark.parametrize("precision", [ssa.SSA_PREC_F64, ssa.SSA_PREC_F32C])
def test_noalloc_matches_plan_two_calls_in_a_row(precision):
    rng = np.random.default_rng(11)
    tol = TOL if precision == ssa.SSA_PREC_F64 else TOL_F32C
    results = []
    for rep in range(2):  # the second pass runs after other calls have reused the array
        for N, L, t in CASES:
            f = synth.many_sines(N, seed=N)
            K = N - L + 1
            x = np.random.default_rng(N + L + t).standard_normal(L if t else K)
            got = _noalloc_product(f, L, x, t, precision)
            ref = _plan_product(f, L, x, t, precision)
            scale = np.linalg.norm(f) * np.linalg.norm(x)
            assert np.max(np.abs(got - ref)) <= tol * scale, (N, L, t)
            results.append(got)
    n = len(CASES)
    for a, b in zip(results[:n], results[n:]):
        np.testing.assert_array_equal(a, b)
    assert rng is not None


def test_noalloc_rejects_oversize_and_host_buffers():
    import torch
    N = 65537
    f = torch.zeros(N, dtype=torch.float64, device="cuda")
    x = torch.zeros(N // 2 + 1, dtype=torch.float64, device="cuda")
    y = torch.zeros(N // 2, dtype=torch.float64, device="cuda")
    with pytest.raises(ssa.SSAError):
        ssa.ssa_matvec_noalloc(f, N, N // 2, 0, x, y)
    fh = np.zeros(100)
    with pytest.raises(ssa.SSAError):
        ssa.ssa_matvec_noalloc(fh, 100, 40, 0, np.zeros(61), np.zeros(40))
