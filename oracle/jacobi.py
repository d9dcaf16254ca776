"""One-sided Jacobi SVD of an explicit matrix (loads the plain-C routine).

Oracle -- test infrastructure only.  Section 2.2 defines the SVD step on the
L x K trajectory matrix (read as X = U Sigma V^T; the printed X = U^T Sigma V
is a typo, since u_i has length L).  ``svd`` returns all min(m, n) triples,
singular values in descending order (section 2.2 orders them that way).
The C source is compiled on first use with the system gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "jacobi_svd.c")
_LIB = os.path.join(_HERE, "c", "_build", "liboracle_jacobi.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C code (plain gcc -O2, no target-specific flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_LIB))
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_jacobi_svd.restype = ctypes.c_int
        lib.oracle_jacobi_svd.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        _lib = lib
    return _lib


def svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 200):
    """Thin SVD A = U diag(s) V^T by one-sided Jacobi, s descending.

    Works on the side with fewer columns: for m < n it factors A^T and swaps.
    Columns of U for zero singular values are left as zeros.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n:
        Ut, s, Vt = svd(A.T, tol, max_sweeps)
        return Vt, s, Ut
    work = np.array(A, dtype=np.float64, order="F", copy=True)
    W = np.zeros((n, n), dtype=np.float64, order="F")
    sweeps = _load().oracle_jacobi_svd(m, n, work.ctypes.data, W.ctypes.data, tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("one-sided Jacobi did not converge")
    s = np.sqrt(np.einsum("ij,ij->j", work, work))
    order = np.argsort(-s, kind="stable")
    s = s[order]
    work = work[:, order]
    W = W[:, order]
    U = np.zeros_like(work)
    nz = s > 0
    U[:, nz] = work[:, nz] / s[nz]
    return U, s, W
