"""Thin ctypes binding of libparac's C ABI (include/parac.h).

Functions carry the C entry points' names and only marshal arguments: numpy
arrays are passed as host pointers, torch CUDA tensors as device pointers; all
computation happens in libparac.so.  Importing this module loads the library
and raises if it has not been built (there is no fallback path).
"""
import ctypes as C
import json
import os

import numpy as np

from . import LIB_PATH

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libparac.so is not built ({LIB_PATH}); run paper_2505_02977_gb300.build.build()")

_lib = C.CDLL(LIB_PATH)

STATUS = {0: "PARAC_OK", 1: "PARAC_EINVAL", 2: "PARAC_ENOT_SDD", 3: "PARAC_ENOMEM", 4: "PARAC_EPOOL",
          5: "PARAC_ETIMEOUT", 6: "PARAC_ECUDA", 7: "PARAC_ENOCONV"}
KIND_AUTO, KIND_LAPLACIAN, KIND_SDDM = 0, 1, 2


class parac_opts(C.Structure):
    _fields_ = [("kind", C.c_int32), ("g_precision", C.c_int32), ("pool_mult", C.c_double),
                ("max_pool_regrow", C.c_int32), ("warps_per_block", C.c_int32), ("spin_limit", C.c_int64),
                ("blocks", C.c_int32), ("queue_chunk", C.c_int32), ("big_threshold", C.c_int32),
                ("sptrsv", C.c_int32), ("check_every", C.c_int32), ("timing", C.c_int32),
                ("stream", C.c_void_p), ("samples", C.c_int32), ("fill_store", C.c_int32),
                ("block_cap", C.c_int32), ("coop", C.c_int32), ("sample_sort", C.c_int32), ("idle_ns", C.c_int32),
                ("trace_path", C.c_char_p), ("trsv_blocks", C.c_int32), ("poll_ns", C.c_int32),
                ("pcg_graph", C.c_int32), ("pcg_many", C.c_int32), ("pcg_workers", C.c_int32),
                ("order", C.c_int32), ("grid_help", C.c_int32), ("grid_help_min", C.c_int32),
                ("host_tables", C.c_int32)]

DEFAULT, ON, OFF = 0, 1, 2
ORDER_GIVEN, ORDER_NNZ = 0, 1
SPTRSV_AUTO, SPTRSV_WARP, SPTRSV_SUB8, SPTRSV_SUB4, SPTRSV_THREAD = 0, 1, 2, 3, 4


class parac_system(C.Structure):
    _fields_ = [("n", C.c_int64), ("colptr", C.c_void_p), ("rowind", C.c_void_p), ("val", C.c_void_p),
                ("ordering", C.c_void_p)]


_lib.parac_opts_default.argtypes = [C.POINTER(parac_opts)]
_lib.parac_factor.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                              C.POINTER(parac_opts), C.POINTER(C.c_void_p)]
_lib.parac_factor.restype = C.c_int
_lib.parac_pcg.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                           C.c_int64, C.c_double, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
_lib.parac_pcg.restype = C.c_int
_lib.parac_factor_many.argtypes = [C.c_int32, C.POINTER(parac_system), C.c_uint64, C.POINTER(parac_opts),
                                   C.POINTER(C.c_void_p)]
_lib.parac_factor_many.restype = C.c_int
_lib.parac_factor_export.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]
_lib.parac_factor_export.restype = C.c_int
_lib.parac_factor_stats.argtypes = [C.c_void_p, C.c_char_p, C.c_size_t]
_lib.parac_factor_stats.restype = C.c_int
_lib.parac_factor_free.argtypes = [C.c_void_p]
_lib.parac_factor_free.restype = None
_lib.parac_precond_apply.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
_lib.parac_precond_apply.restype = C.c_int
_lib.parac_precond_apply_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
_lib.parac_precond_apply_noalloc.restype = C.c_int
_lib.parac_status_string.argtypes = [C.c_int]
_lib.parac_status_string.restype = C.c_char_p
_lib.parac_last_error.argtypes = []
_lib.parac_last_error.restype = C.c_char_p
_lib.parac_autotune.argtypes = [C.c_int32, C.POINTER(parac_system), C.c_uint64, C.POINTER(parac_opts),
                                C.POINTER(parac_opts), C.c_char_p, C.c_size_t]
_lib.parac_autotune.restype = C.c_int
_lib.parac_pcg_many.argtypes = [C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.c_double, C.c_int32, C.c_void_p, C.c_void_p]
_lib.parac_pcg_many.restype = C.c_int
_lib.parac_kernel_launches.argtypes = []
_lib.parac_kernel_launches.restype = C.c_uint64

EXPORTED = ("parac_opts_default", "parac_factor", "parac_pcg", "parac_factor_many", "parac_factor_export",
            "parac_factor_stats", "parac_factor_free", "parac_precond_apply", "parac_status_string",
            "parac_last_error", "parac_kernel_launches", "parac_precond_apply_noalloc", "parac_autotune",
            "parac_pcg_many")


class ParacError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib.parac_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")
        self.code = code
        self.status = STATUS.get(code, str(code))


def _check(code, where, allow=()):
    if code != 0 and code not in allow:
        raise ParacError(code, where)
    return code


def _ptr(a, dtype):
    """Pointer of a numpy array (host) or torch tensor (host or device); None -> NULL."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):          # torch tensor
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr


def parac_opts_default(**kw):
    o = parac_opts()
    _lib.parac_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream if hasattr(v, "cuda_stream") else int(v)
        if k == "trace_path" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


class Factor:
    """Owning wrapper of a parac_factor_t handle."""

    def __init__(self, handle):
        self.handle = C.c_void_p(handle)

    def free(self):
        if self.handle and self.handle.value:
            _lib.parac_factor_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self):
        return parac_factor_stats(self)

    def export(self):
        return parac_factor_export(self)


def parac_factor(n, colptr, rowind, val, ordering=None, seed=0, opts=None):
    keep = []
    ps = []
    for a, dt in ((colptr, np.int64), (rowind, np.int32), (val, np.float64), (ordering, np.int32)):
        p, k = _ptr(a, dt)
        ps.append(p); keep.append(k)
    h = C.c_void_p()
    _check(_lib.parac_factor(n, *ps, seed, C.byref(opts) if opts is not None else None, C.byref(h)), "parac_factor")
    return Factor(h.value)


def parac_factor_many(systems, seed=0, opts=None):
    """systems: list of (n, colptr, rowind, val, ordering-or-None)."""
    keep = []
    arr = (parac_system * len(systems))()
    for i, (n, cp, ri, va, od) in enumerate(systems):
        ptrs = []
        for a, dt in ((cp, np.int64), (ri, np.int32), (va, np.float64), (od, np.int32)):
            p, k = _ptr(a, dt)
            ptrs.append(p); keep.append(k)
        arr[i] = parac_system(n, *ptrs)
    out = (C.c_void_p * len(systems))()
    _check(_lib.parac_factor_many(len(systems), arr, seed, C.byref(opts) if opts is not None else None, out),
           "parac_factor_many")
    return [Factor(out[i]) for i in range(len(systems))]


def _systems(systems):
    keep = []
    arr = (parac_system * len(systems))()
    for i, (n, cp, ri, va, od) in enumerate(systems):
        ptrs = []
        for a, dt in ((cp, np.int64), (ri, np.int32), (va, np.float64), (od, np.int32)):
            p, k = _ptr(a, dt)
            ptrs.append(p); keep.append(k)
        arr[i] = parac_system(n, *ptrs)
    return arr, keep


def parac_autotune(systems, seed=0, opts=None):
    """Tuned options for systems like these: (opts, report dict)."""
    arr, keep = _systems(systems)
    best = parac_opts()
    buf = C.create_string_buffer(8192)
    _check(_lib.parac_autotune(len(systems), arr, seed, C.byref(opts) if opts is not None else None,
                               C.byref(best), buf, 8192), "parac_autotune")
    return best, json.loads(buf.value.decode())


def parac_pcg(G, n, colptr, rowind, val, B, tol=1e-8, maxit=1000, X=None, nrhs=None, allow_noconv=True):
    """Solve L X = B for nrhs <= 32 right-hand sides (PCG, Sec. V).

    B is an n-vector or an (m, nrhs) array with m >= n (numpy, or a torch CUDA
    tensor); column j is B[:n, j] and m is passed as the leading dimension.
    X, if given, is an (mx, nrhs) Fortran-ordered numpy array or a torch
    tensor of the same layout.  Returns (X, iters, relres, status); X has B's
    kind and shape (n,) or (n, nrhs)."""
    if nrhs is None:
        nrhs = 1 if len(getattr(B, "shape", (n,))) == 1 else B.shape[1]
    if hasattr(B, "data_ptr"):
        import torch
        Bd = B.reshape(-1, 1) if B.dim() == 1 else B
        ldb = Bd.shape[0]
        Bd = Bd.t().contiguous()                     # column-major storage
        if X is None:
            X = torch.empty((nrhs, n), dtype=torch.float64, device=B.device)
            ldx = n
            Xv = X.t()
        else:
            ldx = X.shape[0] if X.dim() > 1 else n
            Xv = X
            X = X.t() if X.dim() > 1 else X
            assert X.is_contiguous()
        pb, kb = Bd.data_ptr(), Bd
        px, kx = X.data_ptr(), X
        Xout = Xv[:n] if nrhs > 1 else Xv.reshape(-1)[:n]
    else:
        Ba = np.asarray(B, np.float64)
        Ba = Ba.reshape(-1, 1) if Ba.ndim == 1 else Ba
        ldb = Ba.shape[0]
        Bc = np.asfortranarray(Ba)
        if X is None:
            X = np.zeros((n, nrhs), np.float64, order="F")
        assert X.flags.f_contiguous and X.dtype == np.float64
        ldx = X.shape[0]
        pb, kb = Bc.ctypes.data, Bc
        px, kx = X.ctypes.data, X
        Xout = X[:n, 0] if nrhs == 1 else X[:n]
    keep = [kb, kx]
    ps = []
    for a, dt in ((colptr, np.int64), (rowind, np.int32), (val, np.float64)):
        p, k = _ptr(a, dt)
        ps.append(p); keep.append(k)
    iters = np.zeros(nrhs, np.int32)
    rel = np.zeros(nrhs, np.float64)
    code = _lib.parac_pcg(G.handle, n, *ps, pb, nrhs, ldb, tol, maxit, px, ldx, iters.ctypes.data, rel.ctypes.data)
    _check(code, "parac_pcg", allow=(7,) if allow_noconv else ())
    return Xout, iters, rel, STATUS[code]


def parac_pcg_many(Gs, bs, tol=1e-8, maxit=1000, xs=None, allow_noconv=True):
    """PCG on several systems at once (one right-hand side each).  bs: list of
    n_s-vectors (numpy or torch CUDA); returns (xs, iters, relres, status)."""
    m = len(Gs)
    if len(bs) != m or (xs is not None and len(xs) != m):
        raise ValueError("parac_pcg_many: one right-hand side (and solution) per handle")
    keep = []
    if xs is None:
        xs = []
        for b in bs:
            if hasattr(b, "data_ptr"):
                import torch
                xs.append(torch.empty_like(b))
            else:
                xs.append(np.zeros(len(b)))
    bp = (C.c_void_p * m)(); xp = (C.c_void_p * m)(); hp = (C.c_void_p * m)()
    for i, (G, b, x) in enumerate(zip(Gs, bs, xs)):
        if hasattr(b, "data_ptr"):
            bp[i] = b.data_ptr(); keep.append(b)
        else:
            bb = np.ascontiguousarray(b, np.float64); keep.append(bb); bp[i] = bb.ctypes.data
        xp[i] = x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        hp[i] = G.handle.value
    iters = np.zeros(m, np.int32); rel = np.zeros(m)
    code = _lib.parac_pcg_many(m, hp, bp, xp, tol, maxit, iters.ctypes.data, rel.ctypes.data)
    _check(code, "parac_pcg_many", allow=(7,) if allow_noconv else ())
    return xs, iters, rel, STATUS[code]


def parac_precond_apply(G, r, z=None):
    if hasattr(r, "data_ptr"):
        import torch
        if z is None:
            z = torch.empty_like(r)
        _check(_lib.parac_precond_apply(G.handle, r.data_ptr(), z.data_ptr()), "parac_precond_apply")
        return z
    r = np.ascontiguousarray(r, np.float64)
    z = np.zeros_like(r) if z is None else z
    _check(_lib.parac_precond_apply(G.handle, r.ctypes.data, z.ctypes.data), "parac_precond_apply")
    return z


def parac_precond_apply_noalloc(G, r, z):
    """Allocation-free z = M^{-1} r; r and z are torch CUDA tensors (device memory)."""
    _check(_lib.parac_precond_apply_noalloc(G.handle, r.data_ptr(), z.data_ptr()), "parac_precond_apply_noalloc")
    return z


def parac_factor_export(G):
    nnz = C.c_int64()
    _check(_lib.parac_factor_export(G.handle, C.byref(nnz), None, None, None, None), "parac_factor_export")
    st = parac_factor_stats(G)
    n = st["n"]
    cp = np.zeros(n + 1, np.int64); row = np.zeros(max(nnz.value, 1), np.int32)
    val = np.zeros(max(nnz.value, 1)); D = np.zeros(max(n, 1))
    _check(_lib.parac_factor_export(G.handle, C.byref(nnz), cp.ctypes.data, row.ctypes.data, val.ctypes.data,
                                    D.ctypes.data), "parac_factor_export")
    return dict(n=n, colptr=cp, row=row[:nnz.value], val=val[:nnz.value], D=D[:n])


def parac_factor_stats(G):
    buf = C.create_string_buffer(8192)
    _check(_lib.parac_factor_stats(G.handle, buf, 8192), "parac_factor_stats")
    return json.loads(buf.value.decode())


def parac_factor_free(G):
    G.free()


def parac_status_string(code):
    return _lib.parac_status_string(code).decode()


def parac_last_error():
    return _lib.parac_last_error().decode()


def parac_kernel_launches():
    return int(_lib.parac_kernel_launches())
