"""ctypes wrapper around the C oracle (test infrastructure only)."""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rchol_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

KIND_AUTO, KIND_LAPLACIAN, KIND_SDDM = 0, 1, 2
_ERR = {1: "EINVAL", 2: "ENOT_SDD", 3: "ENOMEM"}


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {_ERR.get(code, code)}")
        self.code = code


def build(force=False, extra_flags=(), out=None):
    """Compile rchol_oracle.c into a shared library (plain gcc, FP contraction off)."""
    so = out or _SO
    if not force and out is None and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           *extra_flags, _SRC, "-o", so + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(so + ".tmp", so)
    return so


_lib = None
_lock = threading.Lock()

P = C.POINTER
i64p, i32p, f64p, u64p = P(C.c_int64), P(C.c_int32), P(C.c_double), P(C.c_uint64)


def _declare(L):
    L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
    L.orc_slot_uniform.argtypes = [C.c_uint64] * 4
    L.orc_slot_uniform.restype = C.c_double
    L.orc_slot_uniform_s.argtypes = [C.c_uint64] * 5
    L.orc_slot_uniform_s.restype = C.c_double
    L.orc_suffix_scan.argtypes = [C.c_int64, f64p, f64p]
    L.orc_pick_bruteforce.argtypes = [C.c_int64, f64p, C.c_int64, C.c_double]
    L.orc_pick_bruteforce.restype = C.c_int64
    L.orc_pick_search.argtypes = [C.c_int64, f64p, C.c_int64, C.c_double]
    L.orc_pick_search.restype = C.c_int64
    L.orc_eliminate_one.argtypes = [C.c_int64, i32p, f64p, C.c_uint64, C.c_uint64, C.c_uint64,
                                    i64p, f64p, i32p, f64p, i32p, f64p, i32p, i32p, f64p, i64p]
    L.orc_eliminate_one_k.argtypes = [C.c_int64, i32p, f64p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int,
                                      i64p, f64p, i32p, f64p, i32p, f64p, i32p, i32p, f64p, i64p]
    L.orc_ingest_dims.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, i64p, i64p, P(C.c_int)]
    L.orc_ingest_copy.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, i64p, i32p, f64p]
    L.orc_factor_run.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, C.c_uint64, C.c_uint64,
                                 P(C.c_void_p)]
    L.orc_factor_run_k.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, C.c_uint64, C.c_uint64, C.c_int,
                                   P(C.c_void_p)]
    L.orc_factor_run_ac.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, C.c_uint64, C.c_uint64, C.c_int,
                                    P(C.c_void_p)]
    L.orc_eliminate_one_ac.argtypes = [C.c_int64, i32p, f64p, C.c_uint64, C.c_uint64, C.c_uint64,
                                       i64p, f64p, i64p, i32p, f64p, i32p, f64p, i32p, i32p, f64p, i64p]
    L.orc_factor_tracked.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, C.c_uint64, C.c_uint64,
                                     C.c_uint64, C.c_int, P(C.c_void_p)]
    L.orc_factor_tracked_ac.argtypes = [C.c_int64, i64p, i32p, f64p, i32p, C.c_int, C.c_uint64, C.c_uint64,
                                        C.c_uint64, C.c_int, C.c_int, P(C.c_void_p)]
    L.orc_factor_dims.argtypes = [C.c_void_p, i64p, i64p, i64p]
    L.orc_factor_copy.argtypes = [C.c_void_p, i64p, i32p, f64p, f64p]
    L.orc_factor_free.argtypes = [C.c_void_p]
    L.orc_dp_update.argtypes = [i32p, C.c_int64, i32p, i32p, C.c_int64, i32p, i32p, i32p, C.c_int]
    L.orc_dp_update.restype = C.c_int64
    L.orc_precond_apply.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, i32p, f64p, f64p, f64p]
    L.orc_pcg.argtypes = [C.c_int64, i64p, i32p, f64p, i64p, i32p, f64p, f64p, i32p, f64p,
                          C.c_double, C.c_int32, f64p, i32p, f64p]
    L.orc_precond_apply32.argtypes = [C.c_int64, i64p, i32p, f64p, f64p, i32p, f64p, f64p, f64p]
    L.orc_pcg_prec.argtypes = [C.c_int64, i64p, i32p, f64p, i64p, i32p, f64p, f64p, i32p, f64p,
                               C.c_double, C.c_int32, C.c_int, f64p, i32p, f64p]


def lib(path=None):
    """Load (building if needed) the oracle library; ``path`` loads a variant build."""
    global _lib
    if path is not None:
        L = C.CDLL(path)
        _declare(L)
        return L
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            _declare(L)
            _lib = L
    return _lib


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(P(t))


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def philox4x64_10(ctr, key, L=None):
    L = L or lib()
    c = _arr(ctr, np.uint64); k = _arr(key, np.uint64); o = np.zeros(4, np.uint64)
    L.orc_philox4x64_10(_p(c, C.c_uint64), _p(k, C.c_uint64), _p(o, C.c_uint64))
    return o


def slot_uniform(seed, k, p, sys=0, q=0, L=None):
    """Uniform of sample q of slot p (q > 0 only for per-slot multi-sampling MS(k))."""
    L = L or lib()
    return L.orc_slot_uniform(seed, k, p, sys) if q == 0 else L.orc_slot_uniform_s(seed, k, p, sys, q)


def suffix_scan(w, L=None):
    L = L or lib()
    w = _arr(w, np.float64); S = np.zeros_like(w)
    L.orc_suffix_scan(len(w), _p(w, C.c_double), _p(S, C.c_double))
    return S


def pick_bruteforce(S, lo, R, L=None):
    L = L or lib()
    S = _arr(S, np.float64)
    return L.orc_pick_bruteforce(len(S), _p(S, C.c_double), lo, R)


def pick_search(S, lo, R, L=None):
    """Search through the exact suffix-maximum envelope of S (as the factor does)."""
    L = L or lib()
    S = _arr(S, np.float64)
    M = np.maximum.accumulate(S[::-1])[::-1].copy()
    return L.orc_pick_search(len(S), _p(M, C.c_double), lo, R)


def eliminate_one(rows, w, seed, k, sys=0, samples=1, L=None):
    """Eliminate one pivot from its gathered entries; returns a dict.  With
    samples > 1 (per-slot multi-sampling MS(samples)) the sampled edges are listed sample by sample:
    sample q of slot p at q*(d-1) + p-1."""
    L = L or lib()
    rows = _arr(rows, np.int32); w = _arr(w, np.float64)
    g = len(rows); m = max(g, 1); ms = m * samples
    d = C.c_int64(); D = C.c_double()
    mrow = np.zeros(m, np.int32); mw = np.zeros(m); mmult = np.zeros(m, np.int32); fval = np.zeros(m)
    slo = np.zeros(ms, np.int32); shi = np.zeros(ms, np.int32); sc = np.zeros(ms); spick = np.zeros(ms, np.int64)
    args = (_p(mrow, C.c_int32), _p(mw, C.c_double), _p(mmult, C.c_int32), _p(fval, C.c_double),
            _p(slo, C.c_int32), _p(shi, C.c_int32), _p(sc, C.c_double), _p(spick, C.c_int64))
    if samples == 1:
        rc = L.orc_eliminate_one(g, _p(rows, C.c_int32), _p(w, C.c_double), seed, k, sys, C.byref(d),
                                 C.byref(D), *args)
    else:
        rc = L.orc_eliminate_one_k(g, _p(rows, C.c_int32), _p(w, C.c_double), seed, k, sys, samples, C.byref(d),
                                   C.byref(D), *args)
    if rc:
        raise OracleError(rc)
    dd = d.value
    ns = max(dd - 1, 0) * samples
    return dict(d=dd, D=D.value, rows=mrow[:dd].copy(), w=mw[:dd].copy(), mult=mmult[:dd].copy(),
                fval=fval[:dd].copy(), lo=slo[:ns].copy(), hi=shi[:ns].copy(), c=sc[:ns].copy(),
                pick=spick[:ns].copy())


def eliminate_one_ac(rows, w, seed, k, sys=0, L=None):
    """One AC(k) pivot on gathered entries (orc_eliminate_one_ac): merged rows
    and F column as eliminate_one; one slot per entry in (weight bits, row)
    order, c[p-1] the weight of slot p, lo = hi = -1 where its sample is a
    self-loop."""
    L = L or lib()
    rows = _arr(rows, np.int32); w = _arr(w, np.float64)
    g = len(rows); m = max(g, 1)
    d = C.c_int64(); D = C.c_double(); ns = C.c_int64()
    mrow = np.zeros(m, np.int32); mw = np.zeros(m); mmult = np.zeros(m, np.int32); fval = np.zeros(m)
    slo = np.zeros(m, np.int32); shi = np.zeros(m, np.int32); sc = np.zeros(m); spick = np.zeros(m, np.int64)
    rc = L.orc_eliminate_one_ac(g, _p(rows, C.c_int32), _p(w, C.c_double), seed, k, sys, C.byref(d), C.byref(D),
                                C.byref(ns), _p(mrow, C.c_int32), _p(mw, C.c_double), _p(mmult, C.c_int32),
                                _p(fval, C.c_double), _p(slo, C.c_int32), _p(shi, C.c_int32), _p(sc, C.c_double),
                                _p(spick, C.c_int64))
    if rc:
        raise OracleError(rc)
    dd, nn = d.value, ns.value
    return dict(d=dd, D=D.value, rows=mrow[:dd].copy(), w=mw[:dd].copy(), mult=mmult[:dd].copy(),
                fval=fval[:dd].copy(), lo=slo[:nn].copy(), hi=shi[:nn].copy(), c=sc[:nn].copy(),
                pick=spick[:nn].copy())


def ingest(colptr, rowind, val, ordering=None, kind=KIND_AUTO, L=None):
    L = L or lib()
    colptr = _arr(colptr, np.int64); rowind = _arr(rowind, np.int32); val = _arr(val, np.float64)
    ordp = None if ordering is None else _arr(ordering, np.int32)
    n = len(colptr) - 1
    nl = C.c_int64(); nnz = C.c_int64(); gr = C.c_int()
    rc = L.orc_ingest_dims(n, _p(colptr, C.c_int64), _p(rowind, C.c_int32), _p(val, C.c_double),
                           _p(ordp, C.c_int32), kind, C.byref(nl), C.byref(nnz), C.byref(gr))
    if rc:
        raise OracleError(rc)
    cp = np.zeros(nl.value + 1, np.int64); row = np.zeros(max(nnz.value, 1), np.int32)
    w = np.zeros(max(nnz.value, 1))
    rc = L.orc_ingest_copy(n, _p(colptr, C.c_int64), _p(rowind, C.c_int32), _p(val, C.c_double),
                           _p(ordp, C.c_int32), kind, _p(cp, C.c_int64), _p(row, C.c_int32), _p(w, C.c_double))
    if rc:
        raise OracleError(rc)
    return dict(n=nl.value, ground=bool(gr.value), colptr=cp, row=row[:nnz.value], w=w[:nnz.value])


def _collect(L, h):
    n = C.c_int64(); nnz = C.c_int64(); st = np.zeros(6, np.int64)
    L.orc_factor_dims(h, C.byref(n), C.byref(nnz), _p(st, C.c_int64))
    cp = np.zeros(n.value + 1, np.int64); row = np.zeros(max(nnz.value, 1), np.int32)
    val = np.zeros(max(nnz.value, 1)); D = np.zeros(max(n.value, 1))
    L.orc_factor_copy(h, _p(cp, C.c_int64), _p(row, C.c_int32), _p(val, C.c_double), _p(D, C.c_double))
    L.orc_factor_free(h)
    return dict(n=n.value, colptr=cp, row=row[:nnz.value], val=val[:nnz.value], D=D[:n.value],
                nnz_low_in=int(st[0]), fill=int(st[1]), nnz_all=int(st[2]), max_gather=int(st[3]),
                depth=int(st[4]), violations=int(st[5]))


def factor(colptr, rowind, val, ordering=None, seed=0, sys=0, kind=KIND_AUTO, samples=1, ac=0, L=None):
    """Sequential rchol factor L ~ F D F^T in label space (Alg. 1 + Alg. 2;
    samples > 1: per-slot multi-sampling MS(samples), every clique-tree slot
    drawing that many edges -- not Sec. VI's AC(2); ac = k >= 1: AC(k), the
    input's entries split into k parallel entries and the elimination run on
    the multigraph, one clique-tree slot per entry, see orc_eliminate_ac)."""
    L = L or lib()
    colptr = _arr(colptr, np.int64); rowind = _arr(rowind, np.int32); val = _arr(val, np.float64)
    ordp = None if ordering is None else _arr(ordering, np.int32)
    h = C.c_void_p()
    if ac:
        if samples != 1:
            raise ValueError("AC(k) takes one sample per slot")
        rc = L.orc_factor_run_ac(len(colptr) - 1, _p(colptr, C.c_int64), _p(rowind, C.c_int32),
                                 _p(val, C.c_double), _p(ordp, C.c_int32), kind, seed, sys, ac, C.byref(h))
    elif samples == 1:
        rc = L.orc_factor_run(len(colptr) - 1, _p(colptr, C.c_int64), _p(rowind, C.c_int32),
                              _p(val, C.c_double), _p(ordp, C.c_int32), kind, seed, sys, C.byref(h))
    else:
        rc = L.orc_factor_run_k(len(colptr) - 1, _p(colptr, C.c_int64), _p(rowind, C.c_int32),
                                _p(val, C.c_double), _p(ordp, C.c_int32), kind, seed, sys, samples, C.byref(h))
    if rc:
        raise OracleError(rc)
    return _collect(L, h)


def factor_tracked(colptr, rowind, val, ordering=None, seed=0, sys=0, kind=KIND_AUTO, sched_seed=1,
                   check=True, ac=0, L=None):
    """Counter-scheduled factor (Sec. III) with a random pick among ready
    vertices (ac = k >= 1: the AC(k) multigraph elimination, see factor)."""
    L = L or lib()
    colptr = _arr(colptr, np.int64); rowind = _arr(rowind, np.int32); val = _arr(val, np.float64)
    ordp = None if ordering is None else _arr(ordering, np.int32)
    h = C.c_void_p()
    rc = L.orc_factor_tracked_ac(len(colptr) - 1, _p(colptr, C.c_int64), _p(rowind, C.c_int32),
                                 _p(val, C.c_double), _p(ordp, C.c_int32), kind, seed, sys, sched_seed,
                                 1 if check else 0, ac, C.byref(h))
    if rc:
        raise OracleError(rc)
    return _collect(L, h)


def dp_update(dp, samples, nbrs, mults, deletes_first=False, L=None):
    L = L or lib()
    dp = _arr(dp, np.int32).copy()
    s = np.asarray(samples, np.int32).reshape(-1, 2)
    sa = np.ascontiguousarray(s[:, 0]); sb = np.ascontiguousarray(s[:, 1])
    nb = _arr(nbrs, np.int32); mu = _arr(mults, np.int32)
    enq = np.zeros(max(len(nb), 1), np.int32)
    ne = L.orc_dp_update(_p(dp, C.c_int32), len(sa), _p(sa, C.c_int32), _p(sb, C.c_int32), len(nb),
                         _p(nb, C.c_int32), _p(mu, C.c_int32), _p(enq, C.c_int32), 1 if deletes_first else 0)
    return dp, enq[:ne].copy()


def precond_apply(F, ordering, r, prec=64, bound=False, L=None):
    """z = P^T F^{-T} D^+ F^{-1} P r.  prec=32: the mixed form (F and the
    solves in FP32, D^+ in FP64; readings M1-M5 of rchol_oracle.c).  With
    bound=True (prec=32 only) also returns the componentwise bound on
    |z - z_exact| that holds for any summation order of the FP32 sums."""
    if prec == 32:
        return _precond_apply32(F, ordering, r, bound, L)
    if prec != 64:
        raise ValueError("prec must be 64 or 32")
    L = L or lib()
    n = F["n"]
    r = _arr(r, np.float64); z = np.zeros(n); work = np.zeros(max(n, 1))
    ordp = None if ordering is None else _arr(ordering, np.int32)
    L.orc_precond_apply(n, _p(F["colptr"], C.c_int64), _p(_arr(F["row"], np.int32), C.c_int32),
                        _p(_arr(F["val"], np.float64), C.c_double), _p(_arr(F["D"], np.float64), C.c_double),
                        _p(ordp, C.c_int32), _p(r, C.c_double), _p(z, C.c_double), _p(work, C.c_double))
    return z


def _precond_apply32(F, ordering, r, bound, L):
    L = L or lib()
    n = F["n"]
    r = _arr(r, np.float64); z = np.zeros(n); bd = np.zeros(max(n, 1)) if bound else None
    ordp = None if ordering is None else _arr(ordering, np.int32)
    rc = L.orc_precond_apply32(n, _p(F["colptr"], C.c_int64), _p(_arr(F["row"], np.int32), C.c_int32),
                               _p(_arr(F["val"], np.float64), C.c_double),
                               _p(_arr(F["D"], np.float64), C.c_double), _p(ordp, C.c_int32),
                               _p(r, C.c_double), _p(z, C.c_double), _p(bd, C.c_double))
    if rc:
        raise OracleError(rc)
    return (z, bd[:n].copy()) if bound else z


def pcg(colptr, rowind, val, F, ordering, b, tol=1e-8, maxit=1000, prec=64, L=None):
    """Oracle PCG with FP64 recurrences, the factor applied in FP64 (prec=64)
    or in the mixed FP32 form (prec=32); returns (x, iterations, true
    relative residual)."""
    L = L or lib()
    colptr = _arr(colptr, np.int64); rowind = _arr(rowind, np.int32); val = _arr(val, np.float64)
    n = len(colptr) - 1
    b = _arr(b, np.float64); x = np.zeros(n)
    ordp = None if ordering is None else _arr(ordering, np.int32)
    it = C.c_int32(); rr = C.c_double()
    rc = L.orc_pcg_prec(n, _p(colptr, C.c_int64), _p(rowind, C.c_int32), _p(val, C.c_double),
                        _p(F["colptr"], C.c_int64), _p(_arr(F["row"], np.int32), C.c_int32),
                        _p(_arr(F["val"], np.float64), C.c_double), _p(_arr(F["D"], np.float64), C.c_double),
                        _p(ordp, C.c_int32), _p(b, C.c_double), tol, maxit, prec, _p(x, C.c_double),
                        C.byref(it), C.byref(rr))
    if rc:
        raise OracleError(rc)
    return x, it.value, rr.value
