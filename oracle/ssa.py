"""Oracle front-ends: decompose a series and reconstruct grouped components.

Oracle -- test infrastructure only.

decompose(f, L, k):  leading k singular triples of the L-trajectory matrix
    (sections 2.1-2.2).  method="jacobi" forms X and runs one-sided Jacobi
    (small N); method="lanczos" runs the oracle's GKL on Algorithms 2/3, whose
    FFTs are the oracle's own radix-2 (fft="radix2") or numpy's (fft="library",
    for the largest sizes; the two are pinned to each other by a test).
    If L > K the K-trajectory matrix (= X^T) is decomposed and U, V swapped
    (the paper assumes L <= K without loss of generality).
    Sign rule (the SVD fixes each pair (u_i, v_i) only up to a common sign):
    flip both so the entry of largest magnitude of u_i is positive, lowest
    index first on ties.
reconstruct(N, L, sigma, U, V, groups):  for each index group I, the
    diagonal average of X_I = sum_{i in I} sigma_i u_i v_i^T (sections 2.3-2.4):
    method="naive" forms X_I and applies the three-case formula,
    method="fft" sums Algorithm 4 over the group, on the oracle's own FFT or,
    with fft="library", on numpy's (the full-size checks; pinned to "radix2").
"""
from __future__ import annotations

import numpy as np

from . import fast_hankel, jacobi, lanczos, trajectory


def validate(N: int, L: int, k: int):
    if N <= 2:
        raise ValueError("need N > 2")
    if not (1 < L < N):
        raise ValueError("need 1 < L < N")
    K = N - L + 1
    if not (1 <= k <= min(L, K)):
        raise ValueError("need 1 <= k <= min(L, K)")


def sign_rule(U: np.ndarray, V: np.ndarray):
    U = U.copy()
    V = V.copy()
    for i in range(U.shape[1]):
        j = int(np.argmax(np.abs(U[:, i])))
        if U[j, i] < 0:
            U[:, i] = -U[:, i]
            V[:, i] = -V[:, i]
    return U, V


def decompose(f, L: int, k: int, method: str = "auto", tol: float = 1e-14, seed: int = 0,
              max_restarts: int = 200, d: int | None = None, max_steps: int | None = None,
              fft: str = "radix2"):
    f = np.asarray(f, dtype=np.float64)
    N = f.size
    validate(N, L, k)
    K = N - L + 1
    if L > K:
        out = decompose(f, K, k, method, tol, seed, max_restarts, d, max_steps, fft)
        U, V = sign_rule(out["V"], out["U"])
        out.update(U=U, V=V)
        return out
    if method == "auto":
        method = "jacobi" if N <= 1500 else "lanczos"
    if method == "jacobi":
        U, s, V = jacobi.svd(trajectory.trajectory_matrix(f, L))
        U, V = sign_rule(U[:, :k], V[:, :k])
        return {"sigma": s[:k].copy(), "U": U, "V": V, "resid": np.zeros(k), "converged": True,
                "method": "jacobi", "all_sigma": s}
    if method != "lanczos":
        raise ValueError(method)
    M = fast_hankel.fft_length(N)
    chat = fast_hankel.spectrum(f, L, M, fft)
    res = lanczos.gkl_svd(lambda v: fast_hankel.hankel_matvec(chat, N, L, v, fft),
                          lambda u: fast_hankel.hankel_rmatvec(chat, N, L, u, fft),
                          L, K, k, d=d, tol=tol, max_restarts=max_restarts, seed=seed,
                          max_steps=max_steps)
    U, V = sign_rule(res.U, res.V)
    return {"sigma": res.sigma, "U": U, "V": V, "resid": res.resid, "converged": res.converged,
            "method": "lanczos", "restarts": res.restarts, "matvecs": res.matvecs,
            "steps": res.steps, "d": res.d}


def reconstruct(N: int, L: int, sigma, U, V, groups, method: str = "naive", fft: str = "radix2") -> np.ndarray:
    sigma = np.asarray(sigma, dtype=np.float64)
    out = np.zeros((len(groups), N))
    for g, idx in enumerate(groups):
        idx = list(idx)
        if method == "naive":
            Y = (U[:, idx] * sigma[idx]) @ V[:, idx].T
            out[g] = trajectory.diagonal_average(Y)
        elif method == "fft":
            for i in idx:
                out[g] += fast_hankel.rank1_hankelization(sigma[i], U[:, i], V[:, i], fft=fft)
        else:
            raise ValueError(method)
    return out
