"""FP64 CPU oracle for the SSsNAL method of arXiv 1910.01312 (linear C-SVC dual).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the CUDA
library and its binding) never imports this package, and this package imports
nothing from it.

The C-SVC method's arithmetic lives in ``svm_oracle.c`` (plain C, FP64,
single thread); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  ``solve(..., omp=True)`` runs the same source built
with OpenMP on all host cores (the benchmark's all-core CPU baseline); its
results are bit-identical to the single-threaded build's.  Beside it, in FP64 numpy: ``mlp.py`` (the learned
warm start's network), ``rff.py`` (random Fourier features, Sec. 4.3), ``nystrom.py`` (the
Nystrom front-end of the same section) and ``gqp.py`` (the method for the unified QP of eq. (1.5), with the SVR dual of
eq. (1.4) as a case).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsvm_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libsvm_oracle_omp.so")
_lock = threading.Lock()
_libs = {False: None, True: None}

OK, ERR_ARG, ERR_OOM, ERR_NOT_CONVERGED, ERR_NUMERIC, ERR_DEGENERATE = 0, 1, 3, 4, 5, 6


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_outer", C.c_int), ("max_inner", C.c_int),
                ("max_ls", C.c_int), ("sigma0", C.c_double), ("sigma_growth", C.c_double),
                ("sigma_max", C.c_double), ("mu", C.c_double), ("delta", C.c_double),
                ("tau", C.c_double), ("eta", C.c_double), ("newton_form", C.c_int)]


class Result(C.Structure):
    _fields_ = [("objective", C.c_double), ("kkt", C.c_double), ("b", C.c_double),
                ("lam_kkt", C.c_double), ("primal", C.c_double), ("gap", C.c_double),
                ("sigma", C.c_double), ("outer", C.c_int), ("inner_total", C.c_int),
                ("status", C.c_int), ("pad", C.c_int), ("n_free", C.c_int64),
                ("n_upper", C.c_int64), ("n_sv", C.c_int64)]


class Trace(C.Structure):
    _fields_ = [("k", C.c_int), ("inner", C.c_int), ("ls_fail", C.c_int), ("pad", C.c_int),
                ("sigma", C.c_double), ("kkt", C.c_double), ("ytalpha", C.c_double),
                ("amin", C.c_double), ("amax", C.c_double), ("gnorm", C.c_double),
                ("p", C.c_int64)]


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (IEEE semantics, no FMA contraction); with
    omp=True the same source with -fopenmp (all host cores)."""
    out = _LIB_OMP if omp else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", *(["-fopenmp"] if omp else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib(omp: bool = False):
    with _lock:
        if _libs[omp] is None:
            L = C.CDLL(build(omp=omp))
            d, i64, vp, i8p, dp, i64p = C.c_double, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p
            L.orc_matvec.argtypes = [vp, C.c_int, i8p, i64, i64, dp, dp]
            L.orc_rmatvec.argtypes = [vp, C.c_int, i8p, i64, i64, dp, dp, dp]
            L.orc_project.argtypes = [dp, i8p, i64, d, dp, dp]
            L.orc_free_set.argtypes = [dp, i8p, i64, d, d, i64p]
            L.orc_free_set.restype = i64
            L.orc_psi.argtypes = [dp, i64, dp, dp, dp, i64, d]
            L.orc_psi.restype = d
            L.orc_newton_direction.argtypes = [vp, C.c_int, i8p, i64, i64, i64p, i64, d, dp, dp, C.c_int]
            L.orc_kkt.argtypes = [vp, C.c_int, i8p, i64, i64, d, dp, dp, dp]
            L.orc_kkt.restype = d
            L.orc_bias.argtypes = [vp, C.c_int, i8p, i64, i64, dp, dp, dp]
            L.orc_bias.restype = d
            L.orc_primal.argtypes = [vp, C.c_int, i8p, i64, i64, d, dp, d]
            L.orc_primal.restype = d
            L.orc_matvec_csr.argtypes = [vp, vp, vp, C.c_int, i8p, i64, i64, dp, dp]
            L.orc_rmatvec_csr.argtypes = [vp, vp, vp, C.c_int, i8p, i64, i64, dp, dp]
            L.orc_kkt_csr.argtypes = [vp, vp, vp, C.c_int, i8p, i64, i64, d, dp, dp, dp]
            L.orc_kkt_csr.restype = d
            L.orc_default_params.argtypes = [C.POINTER(Params)]
            L.orc_solve.argtypes = [vp, C.c_int, i8p, i64, i64, d, C.POINTER(Params), dp, C.c_int,
                                    dp, C.POINTER(Result), C.POINTER(Trace)]
            _libs[omp] = L
    return _libs[omp]


def omp_threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else the host's cores)."""
    v = os.environ.get("OMP_NUM_THREADS", "")
    return int(v) if v.isdigit() and int(v) > 0 else (os.cpu_count() or 1)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _xarg(X):
    X = np.ascontiguousarray(X)
    if X.dtype == np.float32:
        return X, 1
    return np.ascontiguousarray(X, dtype=np.float64), 0


def _yarg(y):
    return np.ascontiguousarray(y, dtype=np.int8)


def matvec(X, y, v):
    """z = A v with A = Diag(y) X."""
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    v = np.ascontiguousarray(v, dtype=np.float64)
    z = np.empty(n, np.float64)
    assert lib().orc_matvec(_p(X), f32, _p(y), n, q, _p(v), _p(z)) == OK
    return z


def rmatvec(X, y, p, with_scale=False):
    """A' p (q-vector); optionally also sum_i |p_i x_ij| per column."""
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty(q, np.float64)
    sc = np.empty(q, np.float64) if with_scale else None
    assert lib().orc_rmatvec(_p(X), f32, _p(y), n, q, _p(p), _p(out), _p(sc)) == OK
    return (out, sc) if with_scale else out


def project(u, y, C_):
    """Pi_{K cap L}(u) by Algorithm 2; returns (pi, lambda_hat)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    y = _yarg(y)
    pi = np.empty_like(u)
    lam = C.c_double(0.0)
    rc = lib().orc_project(_p(u), _p(y), u.size, float(C_), _p(pi), C.byref(lam))
    assert rc == OK, rc
    return pi, lam.value


def free_set(u, y, C_, lam):
    u = np.ascontiguousarray(u, dtype=np.float64)
    y = _yarg(y)
    J = np.empty(u.size, np.int64)
    p = lib().orc_free_set(_p(u), _p(y), u.size, float(C_), float(lam), _p(J))
    return J[:p].copy()


def psi(v, u, pi, alpha, sigma):
    v = np.ascontiguousarray(v, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    pi = np.ascontiguousarray(pi, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    return lib().orc_psi(_p(v), v.size, _p(u), _p(pi), _p(alpha), u.size, float(sigma))


def newton_direction(X, y, J, sigma, g, form=0):
    """Solve (I + sigma A'PA) dv = -g exactly (form 0 auto, 1 q-form, 2 p-form)."""
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    J = np.ascontiguousarray(J, dtype=np.int64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    dv = np.empty(q, np.float64)
    rc = lib().orc_newton_direction(_p(X), f32, _p(y), n, q, _p(J), J.size, float(sigma),
                                    _p(g), _p(dv), int(form))
    assert rc == OK, rc
    return dv


def kkt(X, y, C_, alpha, with_extras=False):
    """R_KKT of eq. (4.1); with_extras also returns (lambda, A'alpha)."""
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    lam = C.c_double(0.0)
    w = np.empty(q, np.float64)
    r = lib().orc_kkt(_p(X), f32, _p(y), n, q, float(C_), _p(alpha), C.byref(lam), _p(w))
    return (r, lam.value, w) if with_extras else r


def bias(X, y, w):
    """Midpoint of the minimiser interval of the hinge term in b; returns (b, lo, hi)."""
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    lo, hi = C.c_double(0.0), C.c_double(0.0)
    b = lib().orc_bias(_p(X), f32, _p(y), n, q, _p(w), C.byref(lo), C.byref(hi))
    return b, lo.value, hi.value


def primal(X, y, C_, w, b):
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().orc_primal(_p(X), f32, _p(y), n, q, float(C_), _p(w), float(b))


def default_params(**kw) -> Params:
    P = Params()
    lib().orc_default_params(C.byref(P))
    for k, v in kw.items():
        setattr(P, k, v)
    return P


def solve(X, y, C_, alpha0=None, trace=False, omp=False, **kw):
    """Run SSsNAL; returns dict(alpha, w, status, objective, kkt, b, ...).
    omp=True: the OpenMP build on all host cores (same results)."""
    X, f32 = _xarg(X)
    y = _yarg(y)
    n, q = X.shape
    P = default_params(**kw)
    alpha = np.zeros(n, np.float64) if alpha0 is None else np.array(alpha0, dtype=np.float64)
    w = np.zeros(q, np.float64)
    res = Result()
    tr = (Trace * max(P.max_outer, 1))() if trace else None
    st = lib(omp).orc_solve(_p(X), f32, _p(y), n, q, float(C_), C.byref(P), _p(alpha),
                         0 if alpha0 is None else 1, _p(w), C.byref(res),
                         tr if trace else None)
    out = {k: getattr(res, k) for k, _ in Result._fields_ if k != "pad"}
    out["status"] = st
    out["alpha"] = alpha
    out["w"] = w
    if trace:
        out["trace"] = [{k: getattr(tr[i], k) for k, _ in Trace._fields_ if k != "pad"}
                        for i in range(res.outer)]
    return out


def _csrarg(indptr, indices, values):
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    v = np.ascontiguousarray(values)
    if v.dtype != np.float32:
        v = np.ascontiguousarray(v, dtype=np.float64)
    return ip, ix, v, int(v.dtype == np.float32)


def matvec_csr(indptr, indices, values, q, y, v):
    """z = A v for X in CSR form (n = len(indptr) - 1 rows, q columns)."""
    ip, ix, vals, f32 = _csrarg(indptr, indices, values)
    y = _yarg(y)
    n = ip.size - 1
    v = np.ascontiguousarray(v, dtype=np.float64)
    z = np.empty(n, np.float64)
    assert lib().orc_matvec_csr(_p(ip), _p(ix), _p(vals), f32, _p(y), n, int(q), _p(v), _p(z)) == OK
    return z


def rmatvec_csr(indptr, indices, values, q, y, p):
    """A' p for X in CSR form (q-vector)."""
    ip, ix, vals, f32 = _csrarg(indptr, indices, values)
    y = _yarg(y)
    n = ip.size - 1
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty(int(q), np.float64)
    assert lib().orc_rmatvec_csr(_p(ip), _p(ix), _p(vals), f32, _p(y), n, int(q), _p(p), _p(out)) == OK
    return out


def kkt_csr(indptr, indices, values, q, y, C_, alpha, with_extras=False, omp=False):
    """R_KKT of eq. (4.1) for X in CSR form; with_extras also returns
    (lambda, A'alpha).  omp=True: the OpenMP build (same result)."""
    ip, ix, vals, f32 = _csrarg(indptr, indices, values)
    y = _yarg(y)
    n = ip.size - 1
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    lam = C.c_double(0.0)
    w = np.empty(int(q), np.float64)
    r = lib(omp).orc_kkt_csr(_p(ip), _p(ix), _p(vals), f32, _p(y), n, int(q), float(C_), _p(alpha),
                             C.byref(lam), _p(w))
    return (r, lam.value, w) if with_extras else r
