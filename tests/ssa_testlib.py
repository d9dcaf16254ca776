"""Helpers shared by the GPU parity tests: call the CUDA library through the
C ABI with host buffers, and compare against the oracle."""
import math

import numpy as np

import paper_0911_4498_gb300 as ssa


def gpu_decompose(f, L, k, precision=ssa.SSA_PREC_F64, **kw):
    f = np.ascontiguousarray(f, dtype=np.float64)
    N = f.size
    K = N - L + 1
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=precision, **kw))
    try:
        d, rc = ssa.ssa_decompose(plan, f, k)
        try:
            sigma = np.empty(k)
            resid = np.empty(k)
            U = np.empty((k, L))
            V = np.empty((k, K))
            ssa.ssa_decomp_get(d, sigma, U, V, resid)
            info = ssa.ssa_decomp_info(d)
            return {"sigma": sigma, "U": U.T.copy(), "V": V.T.copy(), "resid": resid, "info": info, "rc": rc}
        finally:
            ssa.ssa_decomp_destroy(d)
    finally:
        ssa.ssa_plan_destroy(plan)


def gpu_decompose_reconstruct(f, L, k, groups, precision=ssa.SSA_PREC_F64, **kw):
    f = np.ascontiguousarray(f, dtype=np.float64)
    N = f.size
    K = N - L + 1
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=precision, **kw))
    try:
        d, rc = ssa.ssa_decompose(plan, f, k)
        try:
            sigma = np.empty(k)
            U = np.empty((k, L))
            V = np.empty((k, K))
            ssa.ssa_decomp_get(d, sigma, U, V, None)
            off, idx = ssa.groups_csr(groups)
            out = np.empty((len(groups), N))
            ssa.ssa_reconstruct(d, off, idx, len(groups), out)
            return {"sigma": sigma, "U": U.T.copy(), "V": V.T.copy(), "rec": out, "rc": rc,
                    "info": ssa.ssa_decomp_info(d)}
        finally:
            ssa.ssa_decomp_destroy(d)
    finally:
        ssa.ssa_plan_destroy(plan)


def gpu_matvec(f, L, x, transpose, precision=ssa.SSA_PREC_F64):
    f = np.ascontiguousarray(f, dtype=np.float64)
    N = f.size
    K = N - L + 1
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    nvec = x.shape[0]
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=precision))
    try:
        ssa.ssa_set_series(plan, f)
        y = np.empty((nvec, K if transpose else L))
        ssa.ssa_matvec(plan, transpose, x, y, nvec)
        return y
    finally:
        ssa.ssa_plan_destroy(plan)


def gpu_spectrum(f, L):
    f = np.ascontiguousarray(f, dtype=np.float64)
    plan = ssa.ssa_embed_plan(f.size, L, None)
    try:
        ssa.ssa_set_series(plan, f)
        M, single = ssa.ssa_plan_info(plan)
        re = np.empty(M // 2 + 1)
        im = np.empty(M // 2 + 1)
        ssa.ssa_get_spectrum(plan, re, im)
        return re + 1j * im, M, single
    finally:
        ssa.ssa_plan_destroy(plan)


def gpu_hankelize(N, L, sigma, U, V, groups, precision=ssa.SSA_PREC_F64):
    K = N - L + 1
    plan = ssa.ssa_embed_plan(N, L, ssa.make_opts(precision=precision))
    try:
        r = len(sigma)
        Uc = np.ascontiguousarray(np.asarray(U).T)   # (r, L) == column-major L x r
        Vc = np.ascontiguousarray(np.asarray(V).T)
        off, idx = ssa.groups_csr(groups)
        out = np.empty((len(groups), N))
        ssa.ssa_hankelize(plan, np.ascontiguousarray(sigma, dtype=np.float64), Uc, L, Vc, K, r, off, idx,
                          len(groups), out)
        return out
    finally:
        ssa.ssa_plan_destroy(plan)


def clusters(sigma, rel_gap=1e-6):
    """Index groups of near-equal singular values (relative gap to sigma_1 below rel_gap)."""
    out, cur = [], [0]
    for i in range(1, len(sigma)):
        if (sigma[i - 1] - sigma[i]) <= rel_gap * sigma[0]:
            cur.append(i)
        else:
            out.append(cur)
            cur = [i]
    out.append(cur)
    return out


def subspace_sin(A, B):
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return math.sqrt(max(0.0, 1.0 - float(np.min(s)) ** 2))


def compare_vectors(Ug, Uo, sigma, tol, rel_gap=1e-6, skip_below=None):
    """Max vector error: |1 - |u_g.u_o|| for isolated triples, principal-angle
    sine for clusters.  Triples with sigma below skip_below are not compared."""
    worst = 0.0
    for cl in clusters(sigma, rel_gap):
        if skip_below is not None and sigma[cl[0]] < skip_below:
            continue
        if len(cl) == 1:
            i = cl[0]
            e = abs(1.0 - abs(float(Ug[:, i] @ Uo[:, i])))
        else:
            e = subspace_sin(Ug[:, cl], Uo[:, cl])
        worst = max(worst, e)
    assert worst <= tol, f"vector error {worst:.3e} > {tol:.1e}"
    return worst
