"""Golub-Kahan-Lanczos truncated SVD with full reorthogonalisation and thick restart.

Oracle -- test infrastructure only.  Follows section 3 of the paper:

  * Algorithm 1 (section 3.1): u_1 = p_0/beta_1;  alpha_j v_j = A^T u_j - beta_j v_{j-1};
    beta_{j+1} u_{j+1} = A v_j - alpha_j u_j, which builds the lower bidiagonal
    B_k with A V_k = U_{k+1} B_k (relation 1) and
    A^T U_{k+1} = V_k B_k^T + alpha_{k+1} v_{k+1} e_{k+1}^T (relation 2).
  * Full reorthogonalisation (section 3.2.2): every new u (v) is orthogonalised
    against all previous u's (v's) by modified Gram-Schmidt, applied twice.
  * Restart (section 3.3): the Krylov dimension is capped at d and the
    iteration restarts from the best Ritz vectors (thick restart).  The paper
    only cites the scheme; the reading used here:
       d  = min(max(2k, k+32), min(L, K)),  keep kk = k + ceil((d-k)/2) pairs.
    With the SVD B = P S Q^T of the projected matrix, the kept Ritz vectors are
    U P[:, :kk] and V Q[:, :kk]; by relation (2) the residual vector v_{c+1}
    carries couplings rho_i = alpha_{c+1} P[r, i], so the new basis is
    [U P_kk] and [V Q_kk, v_{c+1}] with projected matrix [diag(S_kk) | rho],
    and the bidiagonalisation continues from v_{c+1}.
  * Convergence (from relation 2): the residual of Ritz triple i is
    |alpha_{c+1}| * |P[r, i]| (last row of the left singular vectors of B).
    All k wanted triples are converged when each residual <= tol * sigma_1.
  * Breakdown: a new alpha or beta <= 1e-14 * (largest value seen) is
    replaced by a seeded random vector orthogonalised against the basis, with
    coupling 0; if the basis already spans the space the vector is zero.

The projected matrix is kept as a dense array B whose rows index U columns
and whose columns index V columns; every step subtracts the known couplings
(A v_c - U B[:, c] or A^T u_r - V B[r, :]) and then reorthogonalises.  The
projected SVD uses the oracle's one-sided Jacobi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import jacobi
from .rng import uniform_pm1


@dataclass
class LanczosResult:
    sigma: np.ndarray
    U: np.ndarray
    V: np.ndarray
    resid: np.ndarray
    converged: bool
    restarts: int
    matvecs: int
    steps: int
    d: int


def default_dims(L: int, K: int, k: int):
    d = min(max(2 * k, k + 32), min(L, K))
    kk = k + int(math.ceil((d - k) / 2))
    kk = min(kk, max(d - 1, k))
    return d, kk


def _mgs_twice(Q: np.ndarray, ncols: int, w: np.ndarray) -> np.ndarray:
    for _ in range(2):
        for i in range(ncols):
            q = Q[:, i]
            w -= (q @ w) * q
    return w


def gkl_svd(matvec, rmatvec, L: int, K: int, k: int, d: int | None = None, kk: int | None = None,
            tol: float = 1e-14, max_restarts: int = 200, seed: int = 0,
            max_steps: int | None = None) -> LanczosResult:
    """Leading k singular triples of the L x K operator given by matvec / rmatvec.

    ``max_steps`` bounds the number of bidiagonalisation half-steps (used to
    time a bounded sample; the result is then incomplete).
    """
    dd, kd = default_dims(L, K, k)
    d = dd if d is None else d
    kk = kd if kk is None else kk
    U = np.zeros((L, d + 1), order="F")
    V = np.zeros((K, d + 1), order="F")
    B = np.zeros((d + 1, d + 1))
    counters = {"matvecs": 0, "breakdowns": 0, "halfsteps": 0}
    est = [0.0]

    def normalise(Q, ncols, w, dim):
        nrm = float(np.linalg.norm(w))
        if nrm > 1e-14 * est[0] and nrm > 0.0:
            est[0] = max(est[0], nrm)
            return w / nrm, nrm
        counters["breakdowns"] += 1
        if ncols >= dim:
            return np.zeros(dim), 0.0
        z = np.array(uniform_pm1(seed, counters["breakdowns"], dim))
        z0 = float(np.linalg.norm(z))
        z = _mgs_twice(Q, ncols, z)
        zn = float(np.linalg.norm(z))
        if zn <= 1e-8 * z0:
            return np.zeros(dim), 0.0
        return z / zn, 0.0

    p0 = np.array(uniform_pm1(seed, 0, L))
    U[:, 0] = p0 / np.linalg.norm(p0)
    r, c = 1, 0

    def v_side():
        nonlocal c
        w = rmatvec(U[:, r - 1]) - V[:, :c] @ B[r - 1, :c]
        counters["matvecs"] += 1
        w = _mgs_twice(V, c, w)
        v, alpha = normalise(V, c, w, K)
        V[:, c] = v
        B[r - 1, c] = alpha
        c += 1
        counters["halfsteps"] += 1

    def u_side():
        nonlocal r
        w = matvec(V[:, c - 1]) - U[:, :r] @ B[:r, c - 1]
        counters["matvecs"] += 1
        w = _mgs_twice(U, r, w)
        u, beta = normalise(U, r, w, L)
        U[:, r] = u
        B[r, c - 1] = beta
        r += 1
        counters["halfsteps"] += 1

    def budget_left():
        return max_steps is None or counters["halfsteps"] < max_steps

    restarts = 0
    v_side()                       # Algorithm 1, first half of step 1
    while True:
        while c < d + 1 and budget_left():
            u_side()
            v_side()
        Bp = B[:r, :c - 1]
        alpha_res = B[r - 1, c - 1]
        P, s, Q = jacobi.svd(Bp)
        est[0] = max(est[0], float(s[0]) if s.size else 0.0)
        resid = np.abs(alpha_res * P[r - 1, :])
        m = min(k, s.size)
        converged = bool(np.all(resid[:m] <= tol * (s[0] if s.size else 0.0)))
        if converged or restarts >= max_restarts or not budget_left() or kk >= c - 1:
            break
        restarts += 1
        Unew = U[:, :r] @ P[:, :kk]
        Vnew = V[:, :c - 1] @ Q[:, :kk]
        vres = V[:, c - 1].copy()
        rho = alpha_res * P[r - 1, :kk]
        U[:, :] = 0.0
        V[:, :] = 0.0
        U[:, :kk] = Unew
        V[:, :kk] = Vnew
        V[:, kk] = vres
        B[:, :] = 0.0
        B[np.arange(kk), np.arange(kk)] = s[:kk]
        B[:kk, kk] = rho
        r, c = kk, kk + 1
    m = min(k, s.size)
    return LanczosResult(sigma=s[:m].copy(), U=U[:, :r] @ P[:, :m], V=V[:, :c - 1] @ Q[:, :m],
                         resid=resid[:m].copy(), converged=converged, restarts=restarts,
                         matvecs=counters["matvecs"], steps=counters["halfsteps"], d=d)
