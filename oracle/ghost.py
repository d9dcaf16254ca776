"""Lanczos bidiagonalisation without reorthogonalisation, and the Cullum-Willoughby
test that removes its spurious singular values (section 3.2.1).

Oracle -- test infrastructure only.  Section 3.2.1 of the paper notes that in floating
point the Lanczos vectors lose orthogonality, and that without reorthogonalisation the
projected matrix then carries copies of converged singular values and spurious ones
that have to be recognised afterwards.  The reading taken here:

  * the recurrence of Algorithm 1 runs unchanged, with no Gram-Schmidt at all: from
    u_1 = p_0 / ||p_0||, alpha_j v_j = A^T u_j - beta_j v_{j-1} and
    beta_{j+1} u_{j+1} = A v_j - alpha_j u_j, which builds the (s+1) x s lower bidiagonal
    B (alpha_j on the diagonal, beta_{j+1} below it) with A V = U B;
  * the Golub-Kahan tridiagonal of B is the Lanczos matrix of the process started from
    u_1, so the Cullum-Willoughby comparison matrix is B without its first row
    (deleting the first Lanczos vector);
  * a singular value of B that is simple (no other singular value of B within the
    agreement level) and agrees with a singular value of the comparison matrix is
    spurious; a value with copies is genuine and counted once, represented by the copy
    whose Ritz pair has the smallest residual;
  * two values agree when they differ by at most 1e-10 sigma_1; values at or below that
    level are not candidates;
  * the residual of the Ritz pair (sigma_i, p_i, q_i) of B is |alpha_{s+1}| |p_i[s]|
    (relation 2 with the next alpha), the last entry of the left singular vector.
"""
from __future__ import annotations

import numpy as np


def gkl_no_reorth(matvec, rmatvec, p0: np.ndarray, steps: int):
    """Algorithm 1 with no reorthogonalisation for `steps` steps.

    Returns (B, alpha_next, U, V): B is (steps+1) x steps lower bidiagonal, alpha_next
    the next step's alpha (for the residuals), U the steps+1 left and V the steps right
    Lanczos vectors as columns."""
    u = p0 / np.linalg.norm(p0)
    U = [u]
    V = []
    B = np.zeros((steps + 1, steps))
    beta = 0.0
    v_prev = None
    for j in range(steps):
        w = rmatvec(u) if v_prev is None else rmatvec(u) - beta * v_prev
        alpha = float(np.linalg.norm(w))
        v = w / alpha
        B[j, j] = alpha
        z = matvec(v) - alpha * u
        beta = float(np.linalg.norm(z))
        u = z / beta
        B[j + 1, j] = beta
        U.append(u)
        V.append(v)
        v_prev = v
    alpha_next = float(np.linalg.norm(rmatvec(u) - beta * v_prev))
    return B, alpha_next, np.array(U).T, np.array(V).T


def ritz_residuals(B: np.ndarray, alpha_next: float):
    """Singular values of B (descending) and the residual |alpha_next| |P[-1, i]| of each Ritz pair."""
    P, s, _ = np.linalg.svd(B, full_matrices=False)
    return s, np.abs(alpha_next * P[-1, :])


def cullum_willoughby(sigma, sigma_hat, resid, k: int, tol: float):
    """Indices of the k kept values (ascending) and whether all k passed with small residuals.

    sigma: singular values of B, descending; sigma_hat: those of B without its first row;
    resid: residuals of sigma's Ritz pairs.  When fewer than k pass, the largest unused
    indices fill the list and the result is not converged."""
    sigma = [float(x) for x in sigma]
    hat = [float(x) for x in sigma_hat]
    c = len(sigma)
    agree = 1e-10 * sigma[0]
    kept = []
    i = 0
    while i < c and len(kept) < k and sigma[i] > agree:
        # the group of values that agree with sigma[i]
        group = [i]
        while group[-1] + 1 < c and sigma[group[-1] + 1] >= sigma[i] - agree:
            group.append(group[-1] + 1)
        simple = len(group) == 1
        in_hat = any(abs(h - sigma[i]) <= agree for h in hat)
        if not (simple and in_hat):
            best = group[0]
            for t in group[1:]:
                if resid[t] < resid[best]:
                    best = t
            kept.append(best)
        i = group[-1] + 1
    passed = len(kept) == k and all(resid[t] <= tol * sigma[0] for t in kept)
    for t in range(c):
        if len(kept) >= k:
            break
        if t not in kept:
            kept.append(t)
    return sorted(kept), passed
