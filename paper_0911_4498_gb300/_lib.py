"""ctypes binding of libssa_gb300.so (include/ssa.h), argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may
be numpy arrays (host memory) or torch CUDA tensors (device memory) of
float64 (int32 for group arrays); the library detects which.  All compute
happens in the CUDA library; if it is missing this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libssa_gb300.so")

SSA_OK, SSA_EINVAL, SSA_ENOMEM, SSA_ENOCONV = range(4)
SSA_ECUDA, SSA_ENUMERIC = 5, 6
SSA_PREC_F64, SSA_PREC_F32C = 0, 1
SSA_REFINE_OFF, SSA_REFINE_ON = 0, 1
SSA_REORTH_FULL, SSA_REORTH_PRO, SSA_REORTH_NONE = 0, 1, 2


class SsaOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("max_restarts", ctypes.c_int),
                ("krylov_dim", ctypes.c_int), ("keep", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("refine", ctypes.c_int), ("reorth_skip", ctypes.c_double),
                ("reorth", ctypes.c_int), ("grid_cap", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("mem_budget", ctypes.c_int64),
                ("workers", ctypes.c_int), ("batch_workers", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("batch_max_n", ctypes.c_int64), ("grid_cap", ctypes.c_int)]


class ServeInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("converged", ctypes.c_int), ("restarts", ctypes.c_int),
                ("matvecs", ctypes.c_int64), ("batched", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "queued", "running", "mem_in_use",
                                              "mem_peak", "batches", "batched_requests")]


SSA_SERVE_VECTORS = 1


class SSAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lib = None
_VP, _I64, _I, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_SIGS = {
    "ssa_default_opts": (None, [ctypes.POINTER(SsaOpts)]),
    "ssa_embed_plan": (_I, [_I64, _I64, ctypes.POINTER(SsaOpts), ctypes.POINTER(_VP)]),
    "ssa_plan_info": (_I, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I)]),
    "ssa_set_series": (_I, [_VP, _VP]),
    "ssa_get_spectrum": (_I, [_VP, _VP, _VP]),
    "ssa_matvec": (_I, [_VP, _I, _VP, _VP, _I]),
    "ssa_decompose": (_I, [_VP, _VP, _I, ctypes.POINTER(_VP)]),
    "ssa_decomp_info": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(_I64), ctypes.POINTER(_I)]),
    "ssa_decomp_get": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "ssa_reconstruct": (_I, [_VP, _VP, _VP, _I, _VP]),
    "ssa_hankelize": (_I, [_VP, _VP, _VP, _I64, _VP, _I64, _I, _VP, _VP, _I, _VP]),
    "ssa_plan_destroy": (None, [_VP]),
    "ssa_decomp_destroy": (None, [_VP]),
    "ssa_matvec_noalloc": (_I, [_VP, _I64, _I64, _I, _VP, _VP, _I, _VP]),
    "ssa_decompose_batch": (_I, [_I, _VP, _VP, _VP, _VP, ctypes.POINTER(SsaOpts), ctypes.POINTER(_VP)]),
    "ssa_batch_info": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(_I64)]),
    "ssa_batch_get": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "ssa_batch_reconstruct": (_I, [_VP, _VP, _VP, _I, _VP]),
    "ssa_batch_plan": (_I, [_I, _VP, _VP, _VP, ctypes.POINTER(SsaOpts), ctypes.POINTER(_VP)]),
    "ssa_batch_run": (_I, [_VP, _VP]),
    "ssa_batch_wait": (_I, [_VP]),
    "ssa_batch_destroy": (None, [_VP]),
    "ssa_hmatrix": (_I, [_VP, _I64, _I64, _I64, _I64, _VP, _I, ctypes.POINTER(SsaOpts), _VP]),
    "ssa_serve_default_opts": (None, [ctypes.POINTER(ServeOpts)]),
    "ssa_serve_create": (_I, [ctypes.POINTER(ServeOpts), ctypes.POINTER(_VP)]),
    "ssa_serve_submit": (_I, [_VP, _VP, _I64, _I64, _I, _I, ctypes.POINTER(_I64)]),
    "ssa_serve_poll": (_I, [_VP, _I64, _D, ctypes.POINTER(_I)]),
    "ssa_serve_take": (_I, [_VP, _I64, _VP, _VP, _VP, _VP, ctypes.POINTER(ServeInfo)]),
    "ssa_serve_stats": (_I, [_VP, ctypes.POINTER(ServeStats)]),
    "ssa_serve_destroy": (None, [_VP]),
    "ssa_fft_tiling": (_I, [_I, _I64, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ssa_fft_threads": (_I, [_I, _I64, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "ssa_stats_enable": (_I, [_I]),
    "ssa_stats_get": (_I, [ctypes.POINTER(KernelStat), _I, ctypes.POINTER(_I)]),
    "ssa_kernel_launches": (ctypes.c_uint64, []),
    "ssa_fault_inject_alloc": (_I, [_I64]),
    "ssa_cw_filter": (_I, [_VP, _I, _VP, _I, _VP, _I, _D, _VP, ctypes.POINTER(_I)]),
    "ssa_strerror": (ctypes.c_char_p, [_I]),
    "ssa_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0911_4498_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc: int, allow=()):
    if rc != SSA_OK and rc not in allow:
        detail = lib().ssa_last_error().decode(errors="replace")
        raise SSAError(rc, f"{lib().ssa_strerror(rc).decode()}: {detail}")
    return rc


def _ptr(x, dtype=np.float64):
    """Raw pointer of a numpy array or torch tensor (contiguous, right dtype)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"need a C-contiguous {np.dtype(dtype)} array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"need a contiguous {want} tensor")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def ssa_default_opts() -> SsaOpts:
    o = SsaOpts()
    lib().ssa_default_opts(ctypes.byref(o))
    return o


def make_opts(precision=SSA_PREC_F64, tol=0.0, max_restarts=200, krylov_dim=0, keep=0, seed=0, stream=None,
              refine=SSA_REFINE_OFF, reorth_skip=0.0, reorth=0, grid_cap=0):
    o = ssa_default_opts()
    o.precision, o.tol, o.max_restarts = precision, tol, max_restarts
    o.krylov_dim, o.keep, o.seed = krylov_dim, keep, seed
    o.stream = stream
    o.refine = refine
    o.reorth_skip = reorth_skip
    o.reorth = reorth
    o.grid_cap = grid_cap
    return o


def ssa_embed_plan(N: int, L: int, opts: SsaOpts | None = None):
    h = _VP()
    _check(lib().ssa_embed_plan(N, L, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h


def ssa_plan_info(plan):
    M, sc = _I64(), _I()
    _check(lib().ssa_plan_info(plan, ctypes.byref(M), ctypes.byref(sc)))
    return M.value, bool(sc.value)


def ssa_set_series(plan, f):
    _check(lib().ssa_set_series(plan, _ptr(f)))


def ssa_get_spectrum(plan, re, im):
    _check(lib().ssa_get_spectrum(plan, _ptr(re), _ptr(im)))


def ssa_matvec(plan, transpose: int, x, y, nvec: int = 1):
    _check(lib().ssa_matvec(plan, int(transpose), _ptr(x), _ptr(y), nvec))


def ssa_decompose(plan, f, k: int):
    """Returns (decomp handle, status); status is SSA_OK or SSA_ENOCONV."""
    h = _VP()
    rc = _check(lib().ssa_decompose(plan, _ptr(f), k, ctypes.byref(h)), allow=(SSA_ENOCONV,))
    return h, rc


def ssa_decomp_info(d):
    k, conv, rs, kd = _I(), _I(), _I(), _I()
    mv = _I64()
    _check(lib().ssa_decomp_info(d, ctypes.byref(k), ctypes.byref(conv), ctypes.byref(rs), ctypes.byref(mv),
                                 ctypes.byref(kd)))
    return {"k": k.value, "converged": bool(conv.value), "restarts": rs.value, "matvecs": mv.value,
            "krylov_dim": kd.value}


def ssa_decomp_get(d, sigma=None, U=None, V=None, resid=None):
    _check(lib().ssa_decomp_get(d, _ptr(sigma), _ptr(U), _ptr(V), _ptr(resid)))


def ssa_reconstruct(d, grp_off, grp_idx, m: int, out):
    _check(lib().ssa_reconstruct(d, _ptr(grp_off, np.int32), _ptr(grp_idx, np.int32), m, _ptr(out)))


def ssa_hankelize(plan, sigma, U, ldu: int, V, ldv: int, r: int, grp_off, grp_idx, m: int, out):
    _check(lib().ssa_hankelize(plan, _ptr(sigma), _ptr(U), ldu, _ptr(V), ldv, r, _ptr(grp_off, np.int32),
                               _ptr(grp_idx, np.int32), m, _ptr(out)))


def ssa_plan_destroy(plan):
    lib().ssa_plan_destroy(plan)


def ssa_decomp_destroy(d):
    lib().ssa_decomp_destroy(d)


def ssa_matvec_noalloc(f, N: int, L: int, transpose: int, x, y, precision=SSA_PREC_F64, stream=None):
    _check(lib().ssa_matvec_noalloc(_ptr(f), N, L, int(transpose), _ptr(x), _ptr(y), precision, stream))


def ssa_decompose_batch(f, offsets, Ls, ks, opts: SsaOpts | None = None):
    """Returns (batch handle, status); status is SSA_OK or SSA_ENOCONV."""
    h = _VP()
    n = len(Ls)
    rc = _check(lib().ssa_decompose_batch(n, _ptr(f), _ptr(offsets, np.int64), _ptr(Ls, np.int64),
                                          _ptr(ks, np.int32), ctypes.byref(opts) if opts is not None else None,
                                          ctypes.byref(h)), allow=(SSA_ENOCONV,))
    return h, rc


def ssa_batch_info(b, i: int):
    k, conv, rs = _I(), _I(), _I()
    mv = _I64()
    _check(lib().ssa_batch_info(b, i, ctypes.byref(k), ctypes.byref(conv), ctypes.byref(rs), ctypes.byref(mv)))
    return {"k": k.value, "converged": bool(conv.value), "restarts": rs.value, "matvecs": mv.value}


def ssa_batch_get(b, i: int, sigma=None, U=None, V=None, resid=None):
    _check(lib().ssa_batch_get(b, i, _ptr(sigma), _ptr(U), _ptr(V), _ptr(resid)))


def ssa_batch_plan(offsets, Ls, ks, opts: SsaOpts | None = None):
    """Batch plan for repeated runs (ssa_batch_run / ssa_batch_wait)."""
    h = _VP()
    _check(lib().ssa_batch_plan(len(Ls), _ptr(offsets, np.int64), _ptr(Ls, np.int64), _ptr(ks, np.int32),
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h


def ssa_batch_run(b, f):
    _check(lib().ssa_batch_run(b, _ptr(f)))


def ssa_batch_wait(b) -> int:
    return _check(lib().ssa_batch_wait(b), allow=(SSA_ENOCONV,))


def ssa_batch_reconstruct(b, grp_off, grp_idx, m: int, out):
    _check(lib().ssa_batch_reconstruct(b, _ptr(grp_off, np.int32), _ptr(grp_idx, np.int32), m, _ptr(out)))


def ssa_batch_destroy(b):
    lib().ssa_batch_destroy(b)


def ssa_hmatrix(f, L: int, B: int, T: int, I, opts: SsaOpts | None = None, out=None):
    """H-matrix of section 6.4 (rows: base starts 0..N-B, columns: test starts 0..N-T).

    f: float64 numpy array or CUDA tensor; I: 1-based triple indices.  Returns
    (H, status) with status SSA_OK or SSA_ENOCONV."""
    N = int(f.numel() if hasattr(f, "numel") else f.size)
    idx = np.ascontiguousarray(np.asarray(I, dtype=np.int32))
    if out is None:
        out = np.empty((N - B + 1, N - T + 1))
    rc = _check(lib().ssa_hmatrix(_ptr(f), N, L, B, T, idx.ctypes.data, len(idx),
                                  ctypes.byref(opts) if opts is not None else None, _ptr(out)),
                allow=(SSA_ENOCONV,))
    return out, rc


def ssa_serve_default_opts() -> ServeOpts:
    o = ServeOpts()
    lib().ssa_serve_default_opts(ctypes.byref(o))
    return o


def make_serve_opts(**kw) -> ServeOpts:
    o = ssa_serve_default_opts()
    for key, val in kw.items():
        setattr(o, key, val)
    return o


def ssa_serve_create(opts: ServeOpts | None = None):
    h = _VP()
    _check(lib().ssa_serve_create(ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h


def ssa_serve_submit(srv, f, L: int, k: int, outputs: int = 0) -> int:
    """Queue f (host float64 array); returns the request id."""
    rid = _I64()
    _check(lib().ssa_serve_submit(srv, _ptr(f), int(f.size), L, k, outputs, ctypes.byref(rid)))
    return rid.value


def ssa_serve_poll(srv, rid: int, timeout_s: float = 0.0) -> bool:
    done = _I()
    _check(lib().ssa_serve_poll(srv, rid, timeout_s, ctypes.byref(done)))
    return bool(done.value)


def ssa_serve_take(srv, rid: int, sigma=None, U=None, V=None, resid=None):
    """Copy results into the given host arrays; returns (status, info dict)."""
    info = ServeInfo()
    rc = _check(lib().ssa_serve_take(srv, rid, _ptr(sigma), _ptr(U), _ptr(V), _ptr(resid), ctypes.byref(info)),
                allow=(SSA_ENOCONV,))
    return rc, {n: getattr(info, n) for n, _ in ServeInfo._fields_}


def ssa_serve_stats(srv) -> dict:
    st = ServeStats()
    _check(lib().ssa_serve_stats(srv, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in ServeStats._fields_}


def ssa_serve_destroy(srv):
    lib().ssa_serve_destroy(srv)


def ssa_fft_tiling(precision: int, N: int):
    """(columns per CTA of the forward, inverse four-step column pass); 0 = not tuned yet."""
    a, b = _I(), _I()
    _check(lib().ssa_fft_tiling(precision, N, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ssa_fft_threads(precision: int, N: int):
    """(threads per CTA of the forward column, row and inverse column passes); 0 = not tuned yet."""
    a, b, c = _I(), _I(), _I()
    _check(lib().ssa_fft_threads(precision, N, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def ssa_stats_enable(on: bool):
    _check(lib().ssa_stats_enable(1 if on else 0))


def ssa_stats_get():
    """Per-kernel stats as a list of dicts (name, launches, ms, bytes, flops)."""
    arr = (KernelStat * 64)()
    n = _I()
    _check(lib().ssa_stats_get(arr, 64, ctypes.byref(n)))
    return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "ms": arr[i].ms,
             "bytes": arr[i].bytes, "flops": arr[i].flops} for i in range(min(n.value, 64))]


def ssa_kernel_launches() -> int:
    return int(lib().ssa_kernel_launches())


def ssa_fault_inject_alloc(after: int):
    _check(lib().ssa_fault_inject_alloc(after))


def ssa_strerror(code: int) -> str:
    return lib().ssa_strerror(code).decode()


def ssa_last_error() -> str:
    return lib().ssa_last_error().decode()


def groups_csr(groups):
    """CSR arrays (int32 offsets, int32 indices) for a list of index lists."""
    off = np.zeros(len(groups) + 1, dtype=np.int32)
    idx = []
    for g, members in enumerate(groups):
        idx.extend(int(i) for i in members)
        off[g + 1] = len(idx)
    return off, np.array(idx if idx else [0], dtype=np.int32)


def ssa_cw_filter(sigma, sigma_hat, resid, k: int, tol: float):
    """Host-side Cullum-Willoughby selection: (kept indices, converged)."""
    import numpy as np
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    sigma_hat = np.ascontiguousarray(sigma_hat, dtype=np.float64)
    resid = np.ascontiguousarray(resid, dtype=np.float64)
    keep = np.zeros(k, dtype=np.int32)
    conv = _I()
    _check(lib().ssa_cw_filter(sigma.ctypes.data, int(sigma.size), sigma_hat.ctypes.data if sigma_hat.size else None,
                               int(sigma_hat.size), resid.ctypes.data, int(k), float(tol), keep.ctypes.data,
                               ctypes.byref(conv)))
    return keep, bool(conv.value)
