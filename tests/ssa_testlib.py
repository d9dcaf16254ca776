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
    """Sine of the largest principal angle between span(A) and span(B), as the
    2-norm of the part of B's orthonormal basis outside span(A) (accurate for
    tiny angles, where 1 - cos^2 cancels)."""
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    r = qb - qa @ (qa.T @ qb)
    return float(np.linalg.norm(r, 2))


def vec_sin(a, b):
    """Sine of the angle between the lines spanned by a and b (linear in the
    angle, unlike 1 - |a.b|, which is about theta^2 / 2)."""
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    s = np.sign(float(a @ b)) or 1.0
    # |a - s b| = 2 sin(theta / 2) is accurate for tiny angles; sin = that * cos(theta / 2)
    h = float(np.linalg.norm(a - s * b))
    return h * math.sqrt(max(0.0, 1.0 - h * h / 4.0))


def compare_vectors(Ug, Uo, sigma, tol, rel_gap=1e-6, skip_below=None, res_tol=None, sigma_next=None):
    """Max vector error: the sine of the angle between u_g and u_o for isolated
    triples, the largest principal-angle sine for clusters.  Triples with sigma
    below skip_below are not compared.

    res_tol: a triple whose Ritz residual is at most res_tol * sigma_1 can be
    off by sin(theta) <= res_tol * sigma_1 / gap (Wedin's sin-theta bound, gap
    to the nearest other singular value, sigma_next being the first one not
    returned); each triple or cluster is then allowed max(tol, that bound)."""
    worst = 0.0
    sig = np.asarray(sigma, dtype=np.float64)
    ext = np.append(sig, sigma_next) if sigma_next is not None else sig
    for cl in clusters(sigma, rel_gap):
        if skip_below is not None and sigma[cl[0]] < skip_below:
            continue
        if len(cl) == 1:
            i = cl[0]
            e = vec_sin(Ug[:, i], Uo[:, i])
        else:
            e = subspace_sin(Ug[:, cl], Uo[:, cl])
        allowed = tol
        if res_tol is not None:
            others = np.delete(ext, cl)
            if others.size:
                gap = max(float(np.min(np.abs(others[:, None] - sig[cl][None, :]))), 1e-300)
                allowed = max(tol, res_tol * float(sig[0]) / gap)
        assert e <= allowed, f"vector error {e:.3e} > {allowed:.1e} (triples {cl})"
        worst = max(worst, e / allowed * tol)
    return worst
