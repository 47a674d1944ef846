"""ctypes binding of include/svm_ssnalm.h (argument marshalling only).

Every step of the solver runs in libsvm_ssnalm.so; this module only converts
torch tensors / numpy arrays to pointers and C structs.  It never falls back to
a CPU implementation: if the library is missing it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_NUMERIC, ERR_DEGENERATE, \
    ERR_TIMEOUT, ERR_UNSUPPORTED = range(9)
DENSE_ROWMAJOR, CSR = 0, 1
F32, F64 = 0, 1
PREC_PLAIN_FP64, PREC_MIXED = 0, 1
FORM_FP64_DIRECT, FORM_MIXED, FORM_COMPENSATED, FORM_FP64_CG = range(4)
MEM_DEVICE, MEM_HOST = 0, 1


class Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("q", C.c_int64), ("layout", C.c_int32), ("dtype", C.c_int32),
                ("memory", C.c_int32), ("reserved0", C.c_int32), ("X", C.c_void_p),
                ("indptr", C.c_void_p), ("indices", C.c_void_p), ("values", C.c_void_p),
                ("nnz", C.c_int64), ("y", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("C", C.c_double), ("tol", C.c_double), ("max_outer", C.c_int32),
                ("max_inner", C.c_int32), ("max_ls", C.c_int32), ("precision", C.c_int32),
                ("sigma0", C.c_double), ("sigma_growth", C.c_double), ("sigma_max", C.c_double),
                ("mu", C.c_double), ("delta", C.c_double), ("tau", C.c_double), ("eta", C.c_double),
                ("newton_mode", C.c_int32), ("deterministic", C.c_int32), ("stream", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("alpha", C.c_void_p), ("w", C.c_void_p), ("b", C.c_double), ("kkt", C.c_double),
                ("objective", C.c_double), ("primal_objective", C.c_double), ("gap", C.c_double),
                ("sigma", C.c_double), ("outer_iters", C.c_int32), ("inner_iters_total", C.c_int32),
                ("status", C.c_int32), ("form", C.c_int32), ("n_free", C.c_int64),
                ("n_upper", C.c_int64), ("n_sv", C.c_int64)]


GQP_DENSE, GQP_STACKED = 0, 1


class GqpProblem(C.Structure):
    _fields_ = [("n", C.c_int64), ("q", C.c_int64), ("layout", C.c_int32), ("dtype", C.c_int32),
                ("memory", C.c_int32), ("reserved0", C.c_int32), ("B", C.c_void_p), ("c", C.c_void_p),
                ("a", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p), ("d", C.c_double)]


class GqpResult(C.Structure):
    _fields_ = [("x", C.c_void_p), ("w", C.c_void_p), ("lam", C.c_double), ("kkt", C.c_double),
                ("objective", C.c_double), ("feasibility", C.c_double), ("sigma", C.c_double),
                ("outer_iters", C.c_int32), ("inner_iters_total", C.c_int32), ("status", C.c_int32),
                ("reserved0", C.c_int32), ("n_free", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("matvec_calls", C.c_int64), ("matvec_ms", C.c_double),
                ("rmatvec_calls", C.c_int64), ("rmatvec_ms", C.c_double), ("proj_calls", C.c_int64),
                ("proj_ms", C.c_double), ("newton_calls", C.c_int64), ("newton_ms", C.c_double),
                ("host_syncs", C.c_int64), ("matvec2_calls", C.c_int64), ("matvec2_ms", C.c_double)]


SYMBOLS = ["svm_default_params", "svm_ssnalm_create", "svm_ssnalm_solve", "svm_ssnalm_destroy",
           "svm_ssnalm_last_error", "svm_op_matvec", "svm_op_rmatvec", "svm_op_project",
           "svm_op_newton", "svm_op_kkt", "svm_op_gram", "svm_ssnalm_solve_batch", "svm_rff_features", "svm_ssnalm_set_timing", "svm_ssnalm_get_stats",
           "svm_rmatvec_noalloc", "svm_mlp_create", "svm_mlp_destroy", "svm_mlp_get_params",
           "svm_mlp_features", "svm_mlp_labels", "svm_mlp_gather", "svm_mlp_forward", "svm_mlp_loss_grad", "svm_mlp_adam_step",
           "svm_mlp_train_step", "svm_mlp_start_point", "svm_ssnalm_solve_mlp", "svm_ssnalm_set_warmstart_model",
           "svm_gqp_create", "svm_svr_create", "svm_gqp_solve", "svm_gqp_destroy", "svm_gqp_last_error",
           "svm_gqp_op_project", "svm_gqp_op_newton", "svm_gqp_op_matvec", "svm_gqp_op_rmatvec",
           "svm_nystrom_kmeans", "svm_nystrom_features"]
MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM = 132, 256, 3, 100611

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsvm_ssnalm.so (raises if it is missing and not built here)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
            _build.build()
        L = C.CDLL(_build.LIB)
        vp, i64 = C.c_void_p, C.c_int64
        L.svm_default_params.argtypes = [C.POINTER(Params)]
        L.svm_default_params.restype = None
        L.svm_ssnalm_create.argtypes = [C.POINTER(vp), C.POINTER(Problem), C.POINTER(Params)]
        L.svm_ssnalm_create.restype = C.c_int
        L.svm_ssnalm_solve.argtypes = [vp, vp, C.POINTER(Result)]
        L.svm_ssnalm_solve.restype = C.c_int
        L.svm_ssnalm_destroy.argtypes = [vp]
        L.svm_ssnalm_destroy.restype = None
        L.svm_ssnalm_last_error.argtypes = [vp]
        L.svm_ssnalm_last_error.restype = C.c_char_p
        L.svm_op_matvec.argtypes = [vp, vp, vp]
        L.svm_op_rmatvec.argtypes = [vp, vp, vp]
        L.svm_op_project.argtypes = [vp, vp, vp, C.POINTER(C.c_double), vp, C.POINTER(i64), vp,
                                     C.POINTER(i64)]
        L.svm_op_newton.argtypes = [vp, vp, i64, C.c_double, vp, vp]
        L.svm_op_kkt.argtypes = [vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.svm_op_gram.argtypes = [vp, vp, i64, vp, vp]
        L.svm_ssnalm_solve_batch.argtypes = [vp, C.c_int32, vp, vp, vp, vp, C.POINTER(Result)]
        L.svm_rff_features.argtypes = [vp, i64, i64, vp, i64, vp, vp]
        L.svm_ssnalm_set_timing.argtypes = [vp, C.c_int]
        L.svm_ssnalm_get_stats.argtypes = [vp, C.POINTER(Stats), C.c_int]
        L.svm_rmatvec_noalloc.argtypes = [vp, vp, i64, i64, vp, vp, vp]
        f32, dbl = C.c_float, C.c_double
        L.svm_mlp_create.argtypes = [C.POINTER(vp), vp, i64, vp]
        L.svm_mlp_destroy.argtypes = [vp]
        L.svm_mlp_destroy.restype = None
        L.svm_mlp_get_params.argtypes = [vp, vp]
        L.svm_mlp_features.argtypes = [vp, vp, i64, i64, dbl, vp, vp]
        L.svm_mlp_forward.argtypes = [vp, vp, i64, vp]
        L.svm_mlp_labels.argtypes = [vp, i64, dbl, vp, vp]
        L.svm_mlp_gather.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.svm_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.svm_mlp_adam_step.argtypes = [vp, vp, i64, f32, f32]
        L.svm_mlp_train_step.argtypes = [vp, vp, vp, i64, vp, i64, f32, f32, vp]
        L.svm_mlp_start_point.argtypes = [vp, vp, i64, dbl, vp]
        L.svm_ssnalm_solve_mlp.argtypes = [vp, vp, C.POINTER(Result), C.POINTER(C.c_int32)]
        L.svm_ssnalm_set_warmstart_model.argtypes = [vp, vp]
        L.svm_gqp_create.argtypes = [C.POINTER(vp), C.POINTER(GqpProblem), C.POINTER(Params)]
        L.svm_svr_create.argtypes = [C.POINTER(vp), vp, i64, i64, C.c_int32, C.c_int32, vp, C.c_double,
                                     C.POINTER(Params)]
        L.svm_gqp_solve.argtypes = [vp, C.POINTER(GqpResult)]
        L.svm_gqp_destroy.argtypes = [vp]
        L.svm_gqp_destroy.restype = None
        L.svm_gqp_last_error.argtypes = [vp]
        L.svm_gqp_last_error.restype = C.c_char_p
        L.svm_gqp_op_project.argtypes = [vp, vp, vp, C.POINTER(C.c_double), vp, C.POINTER(i64)]
        L.svm_gqp_op_newton.argtypes = [vp, vp, i64, C.c_double, vp, vp]
        L.svm_gqp_op_matvec.argtypes = [vp, vp, vp]
        L.svm_gqp_op_rmatvec.argtypes = [vp, vp, vp]
        L.svm_nystrom_kmeans.argtypes = [vp, i64, i64, vp, i64, C.c_int32, vp, vp, vp]
        L.svm_nystrom_features.argtypes = [vp, i64, i64, vp, i64, C.c_double, C.c_double, vp, C.c_int32, vp]
        for f in ("svm_op_matvec", "svm_op_rmatvec", "svm_op_project", "svm_op_newton", "svm_op_kkt", "svm_op_gram",
                  "svm_ssnalm_solve_batch", "svm_rff_features",
                  "svm_ssnalm_set_timing", "svm_ssnalm_get_stats", "svm_rmatvec_noalloc", "svm_mlp_create",
                  "svm_mlp_get_params", "svm_mlp_features", "svm_mlp_labels", "svm_mlp_gather", "svm_mlp_forward",
                  "svm_mlp_loss_grad",
                  "svm_mlp_adam_step", "svm_mlp_train_step", "svm_mlp_start_point", "svm_ssnalm_solve_mlp",
                  "svm_ssnalm_set_warmstart_model", "svm_gqp_create", "svm_svr_create", "svm_gqp_solve",
                  "svm_gqp_op_project", "svm_gqp_op_newton", "svm_gqp_op_matvec", "svm_gqp_op_rmatvec",
                  "svm_nystrom_kmeans", "svm_nystrom_features"):
            getattr(L, f).restype = C.c_int
        _lib = L
        return L


class SVMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def default_params(**kw) -> Params:
    P = Params()
    load().svm_default_params(C.byref(P))
    for k, v in kw.items():
        if not hasattr(P, k):
            raise KeyError(k)
        setattr(P, k, v)
    return P


def _check_noalloc_args(X, y, c, out):
    """Types, shapes and devices of svm_rmatvec_noalloc's buffers: the C call
    trusts them, so a wrong one would make the kernel read or write outside a
    buffer.  Raises TypeError / ValueError."""
    for name, t in (("X", X), ("y", y), ("c", c), ("out", out)):
        if not hasattr(t, "data_ptr"):
            raise TypeError(f"{name} must be a torch tensor")
    want = (("X", X, "float32"), ("y", y, "int8"), ("c", c, "float64"), ("out", out, "float64"))
    for name, t, dt in want:
        if not str(t.dtype).endswith(dt):
            raise TypeError(f"{name} must be {dt}, got {t.dtype}")
    if X.dim() != 2:
        raise ValueError("X must be 2-D (n x q)")
    n, q = X.shape
    for name, t, m in (("y", y, n), ("c", c, n), ("out", out, q)):
        if tuple(t.shape) != (m,):
            raise ValueError(f"{name} must have shape ({m},), got {tuple(t.shape)}")
    devs = {(t.device.type, t.device.index) for t in (X, y, c, out)}
    if any(d[0] != "cuda" for d in devs) or len(devs) != 1:
        raise ValueError("X, y, c and out must be CUDA tensors on one device")
    import torch
    if next(iter(devs))[1] != torch.cuda.current_device():
        raise ValueError("the buffers must be on the current CUDA device")


def rmatvec_noalloc(X, y, c, out, stream=None) -> int:
    """out = A'c through the allocation-free entry point (device FP32 X (n x q),
    int8 y (n), FP64 c (n) and out (q), all on the current device); returns the
    svm_status code.  Raises TypeError / ValueError for other buffers."""
    _check_noalloc_args(X, y, c, out)
    n, q = X.shape
    return load().svm_rmatvec_noalloc(_ptr(X), _ptr(y), int(n), int(q), _ptr(c), _ptr(out), stream)


def rff_features(X, Omega, Z, stream=None) -> int:
    """Random Fourier features Z (n x 2N) of X (n x q) for the frequencies
    Omega (q x N), all device FP32; returns the svm_status code."""
    n, q = X.shape
    N = Omega.shape[1]
    return load().svm_rff_features(_ptr(X), int(n), int(q), _ptr(Omega), int(N), _ptr(Z), stream)


def nystrom_kmeans(X, centres, iters, labels=None, stream=None):
    """Lloyd's k-means on the rows of X (device FP32, n x q) from the initial
    centres (device FP64, r x q, updated in place); labels (device int32, n,
    optional) receives the last assignment.  Returns the objective of each
    iteration (numpy array); raises SVMError on failure."""
    n, q = X.shape
    r = centres.shape[0]
    obj = np.zeros(int(iters), np.float64)
    st = load().svm_nystrom_kmeans(_ptr(X), int(n), int(q), _ptr(centres), int(r), int(iters), _ptr(labels),
                                   obj.ctypes.data_as(C.c_void_p), stream)
    if st != OK:
        raise SVMError(st, "svm_nystrom_kmeans")
    return obj


def nystrom_features(X, centres, alpha, Z, shift=1e-3, stream=None):
    """Z = K_nr L^{-T}, L L' = K_rr + shift I (Z device, n x r, FP32 or FP64)."""
    n, q = X.shape
    r = centres.shape[0]
    zd = F32 if str(Z.dtype).endswith("float32") else F64
    st = load().svm_nystrom_features(_ptr(X), int(n), int(q), _ptr(centres), int(r), float(alpha), float(shift),
                                     _ptr(Z), zd, stream)
    if st != OK:
        raise SVMError(st, "svm_nystrom_features")


def _ptr(t):
    """Address of a torch tensor or numpy array (contiguous)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("the C ABI takes contiguous (row-major) tensors")
        return t.data_ptr()
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("the C ABI takes C-contiguous (row-major) arrays")
    return t.ctypes.data


class Solver:
    """Owns one svm_ssnalm_t handle.

    X, y: torch CUDA tensors (memory=DEVICE, borrowed: keep them alive) or
    host arrays -- numpy or torch CPU tensors, pinned or not -- (memory=HOST,
    copied to the device by create; the solve's outputs are then host arrays
    too).  For a sparse X pass csr=(indptr, indices, values, q) instead (same
    memory rules; X is then ignored)."""

    def __init__(self, X, y, C_=1.0, stream=None, csr=None, **params):
        self._lib = load()
        self.h = C.c_void_p()
        if csr is not None:
            # csr = (indptr int64 [n+1], indices int32 [nnz], values FP32/FP64 [nnz], q); X unused
            indptr, indices, values, q = csr
            n, V = int(indptr.shape[0]) - 1, values
        else:
            n, q = X.shape
            V = X
        is_host = not bool(getattr(V, "is_cuda", False))
        self.memory = MEM_HOST if is_host else MEM_DEVICE
        dt = str(V.dtype)
        if dt.endswith("float32"):
            dtype = F32
        elif dt.endswith("float64"):
            dtype = F64
        else:
            raise TypeError(f"X dtype {dt} not supported")
        self.n, self.q = int(n), int(q)
        if csr is not None:
            self._keep = (indptr, indices, values, y)
            prob = Problem(n=n, q=q, layout=CSR, dtype=dtype, memory=self.memory, X=None, indptr=_ptr(indptr),
                           indices=_ptr(indices), values=_ptr(values), nnz=int(values.shape[0]), y=_ptr(y))
        else:
            self._keep = (X, y)
            prob = Problem(n=n, q=q, layout=DENSE_ROWMAJOR, dtype=dtype, memory=self.memory, X=_ptr(X),
                           indptr=None, indices=None, values=None, nnz=0, y=_ptr(y))
        P = default_params(C=float(C_), **params)
        if stream is not None:
            P.stream = stream
        self.params = P
        st = self._lib.svm_ssnalm_create(C.byref(self.h), C.byref(prob), C.byref(P))
        if st != OK:
            raise SVMError(st, self._lib.svm_ssnalm_last_error(None).decode())

    def close(self):
        if self.h:
            self._lib.svm_ssnalm_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._lib.svm_ssnalm_last_error(self.h).decode()

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise SVMError(st, self.last_error())
        return st

    def solve(self, alpha, w, alpha0=None, allow=(OK, ERR_NOT_CONVERGED, ERR_DEGENERATE)):
        """alpha (n), w (q): FP64 output buffers (device tensors or numpy)."""
        R = Result(alpha=_ptr(alpha), w=_ptr(w))
        st = self._lib.svm_ssnalm_solve(self.h, _ptr(alpha0), C.byref(R))
        self._check(st, allow)
        out = {k: getattr(R, k) for k, _ in Result._fields_ if k not in ("alpha", "w")}
        out["status"] = st
        return out

    def solve_batch(self, Y, Cs, alpha, w, allow=(OK, ERR_NOT_CONVERGED, ERR_DEGENERATE)):
        """B problems sharing this handle's X: labels Y (B x n int8), bounds Cs
        (B floats), outputs alpha (B x n FP64) and w (B x q FP64) in the
        handle's memory kind.  Returns (status, [per-problem result dicts])."""
        Cs = np.ascontiguousarray(np.asarray(Cs, dtype=np.float64))
        B = int(Cs.size)
        R = (Result * B)()
        st = self._lib.svm_ssnalm_solve_batch(self.h, B, _ptr(Y), Cs.ctypes.data_as(C.c_void_p), _ptr(alpha),
                                              _ptr(w), R)
        self._check(st, allow)
        outs = []
        for b in range(B):
            outs.append({k: getattr(R[b], k) for k, _ in Result._fields_ if k not in ("alpha", "w")})
        return st, outs

    def solve_mlp(self, mlp, alpha, w, allow=(OK, ERR_NOT_CONVERGED, ERR_DEGENERATE)):
        """Warm-started solve from the network `mlp` (an MLP), cold fallback;
        the returned dict adds "used_warm"."""
        R = Result(alpha=_ptr(alpha), w=_ptr(w))
        used = C.c_int32(0)
        st = self._lib.svm_ssnalm_solve_mlp(self.h, mlp.h, C.byref(R), C.byref(used))
        self._check(st, allow)
        out = {k: getattr(R, k) for k, _ in Result._fields_ if k not in ("alpha", "w")}
        out["status"] = st
        out["used_warm"] = used.value
        return out

    def set_warmstart_model(self, params=None):
        """Attach a trained network (device FP32 parameter vector, copied) so
        that solve() without alpha0 starts from its prediction; None detaches."""
        self._check(self._lib.svm_ssnalm_set_warmstart_model(self.h, _ptr(params)))

    def set_timing(self, enable=True):
        self._check(self._lib.svm_ssnalm_set_timing(self.h, 1 if enable else 0))

    def stats(self, reset=False):
        S = Stats()
        self._check(self._lib.svm_ssnalm_get_stats(self.h, C.byref(S), 1 if reset else 0))
        return {k: getattr(S, k) for k, _ in S._fields_}

    # ---- step-level entry points (device FP64 buffers) ----
    def matvec(self, v, z):
        self._check(self._lib.svm_op_matvec(self.h, _ptr(v), _ptr(z)))

    def rmatvec(self, c, out):
        self._check(self._lib.svm_op_rmatvec(self.h, _ptr(c), _ptr(out)))

    def project(self, u, pi, J=None, S=None):
        lam = C.c_double(0.0)
        p, s = C.c_int64(0), C.c_int64(0)
        self._check(self._lib.svm_op_project(self.h, _ptr(u), _ptr(pi), C.byref(lam), _ptr(J),
                                             C.byref(p), _ptr(S), C.byref(s)))
        return lam.value, p.value, s.value

    def newton(self, J, p, sigma, g, dv):
        self._check(self._lib.svm_op_newton(self.h, _ptr(J), int(p), float(sigma), _ptr(g), _ptr(dv)))

    def gram(self, J, p, G, hsum):
        """G = X_J' X_J (tcgen05 tensor cores, TF32 products) and hsum = X_J' 1."""
        self._check(self._lib.svm_op_gram(self.h, _ptr(J), int(p), _ptr(G), _ptr(hsum)))

    def kkt(self, alpha):
        r, lam = C.c_double(0.0), C.c_double(0.0)
        self._check(self._lib.svm_op_kkt(self.h, _ptr(alpha), C.byref(r), C.byref(lam)))
        return r.value, lam.value


def _mlp_check(st, what):
    if st != OK:
        raise SVMError(st, what)


def mlp_features(X, y, C_, F, stream=None):
    """F (n x 132, FP32) = warm-start features of the device problem (X FP32
    n x 128, y int8)."""
    n, q = X.shape
    _mlp_check(load().svm_mlp_features(_ptr(X), _ptr(y), int(n), int(q), float(C_), _ptr(F), stream),
               "svm_mlp_features")


def mlp_labels(alpha, C_, labels, stream=None):
    """labels (int32) = 0 / 1 / 2 where alpha (FP64) is at 0 / free / at C."""
    _mlp_check(load().svm_mlp_labels(_ptr(alpha), int(alpha.shape[0]), float(C_), _ptr(labels), stream),
               "svm_mlp_labels")


def mlp_gather(F, labels, idx, Fb, Lb, stream=None):
    """Fb[r] = F[idx[r]], Lb[r] = labels[idx[r]] (idx int64 on the device)."""
    _mlp_check(load().svm_mlp_gather(_ptr(F), _ptr(labels), _ptr(idx), int(idx.shape[0]), _ptr(Fb), _ptr(Lb), stream),
               "svm_mlp_gather")


class MLP:
    """Owns one svm_mlp_t (the warm-start network) on a stream; tensors are
    device tensors (FP32 features and parameters, int32 labels)."""

    def __init__(self, params, max_rows, stream=None):
        self._lib = load()
        self.h = C.c_void_p()
        self.max_rows = int(max_rows)
        _mlp_check(self._lib.svm_mlp_create(C.byref(self.h), _ptr(params), self.max_rows, stream), "svm_mlp_create")

    def close(self):
        if self.h:
            self._lib.svm_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, out):
        _mlp_check(self._lib.svm_mlp_get_params(self.h, _ptr(out)), "svm_mlp_get_params")

    def forward(self, F, logits):
        _mlp_check(self._lib.svm_mlp_forward(self.h, _ptr(F), int(F.shape[0]), _ptr(logits)), "svm_mlp_forward")

    def loss_grad(self, F, labels, cw, loss, grad):
        _mlp_check(self._lib.svm_mlp_loss_grad(self.h, _ptr(F), _ptr(labels), int(F.shape[0]), _ptr(cw), _ptr(loss),
                                               _ptr(grad)), "svm_mlp_loss_grad")

    def adam_step(self, grad, t, lr, wd=0.0):
        _mlp_check(self._lib.svm_mlp_adam_step(self.h, _ptr(grad), int(t), float(lr), float(wd)), "svm_mlp_adam_step")

    def train_step(self, F, labels, cw, t, lr, wd=0.0, loss=None):
        _mlp_check(self._lib.svm_mlp_train_step(self.h, _ptr(F), _ptr(labels), int(F.shape[0]), _ptr(cw), int(t),
                                                float(lr), float(wd), _ptr(loss)), "svm_mlp_train_step")

    def start_point(self, F, C_, alpha0):
        _mlp_check(self._lib.svm_mlp_start_point(self.h, _ptr(F), int(F.shape[0]), float(C_), _ptr(alpha0)),
                   "svm_mlp_start_point")


class GQP:
    """Owns one svm_gqp_t: SSsNAL for the unified QP of eq. (1.5),
    min 1/2 x'BB'x + c'x s.t. a'x = d, l <= x <= u.  B (n x q, or X (n/2 x q)
    with stacked=True for B = [X; -X]) and the FP64 vectors c, a, l, u are all
    torch CUDA tensors (borrowed: keep them alive) or all host arrays (copied)."""

    def __init__(self, B, c, a, l, u, d=0.0, stacked=False, stream=None, _h=None, _keep=None, **params):
        self._lib = load()
        self.h = C.c_void_p()
        P = default_params(**params)
        if stream is not None:
            P.stream = stream
        self.params = P
        if _h is not None:           # built by GQP.svr
            self.h, (self.n, self.q, self.memory), self._keep = _h, _keep[0], _keep[1]
            return
        is_host = not bool(getattr(B, "is_cuda", False))
        self.memory = MEM_HOST if is_host else MEM_DEVICE
        dt = str(B.dtype)
        dtype = F32 if dt.endswith("float32") else F64 if dt.endswith("float64") else None
        if dtype is None:
            raise TypeError(f"B dtype {dt} not supported")
        m, q = B.shape
        n = 2 * m if stacked else m
        self.n, self.q = int(n), int(q)
        self._keep = (B, c, a, l, u)
        prob = GqpProblem(n=n, q=q, layout=GQP_STACKED if stacked else GQP_DENSE, dtype=dtype, memory=self.memory,
                          B=_ptr(B), c=_ptr(c), a=_ptr(a), l=_ptr(l), u=_ptr(u), d=float(d))
        st = self._lib.svm_gqp_create(C.byref(self.h), C.byref(prob), C.byref(P))
        if st != OK:
            raise SVMError(st, self._lib.svm_gqp_last_error(None).decode())

    @classmethod
    def svr(cls, X, y, eps, C_, stream=None, **params):
        """The linear SVR dual (eq. (1.4)) over X (m x q) and targets y (FP64, m)."""
        L = load()
        P = default_params(C=float(C_), **params)
        if stream is not None:
            P.stream = stream
        is_host = not bool(getattr(X, "is_cuda", False))
        dt = str(X.dtype)
        dtype = F32 if dt.endswith("float32") else F64 if dt.endswith("float64") else None
        if dtype is None:
            raise TypeError(f"X dtype {dt} not supported")
        m, q = X.shape
        h = C.c_void_p()
        st = L.svm_svr_create(C.byref(h), _ptr(X), int(m), int(q), dtype, MEM_HOST if is_host else MEM_DEVICE,
                              _ptr(y), float(eps), C.byref(P))
        if st != OK:
            raise SVMError(st, L.svm_gqp_last_error(None).decode())
        return cls(None, None, None, None, None, stream=stream, _h=h,
                   _keep=((2 * int(m), int(q), MEM_HOST if is_host else MEM_DEVICE), (X,)), **params)

    def close(self):
        if self.h:
            self._lib.svm_gqp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._lib.svm_gqp_last_error(self.h).decode()

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise SVMError(st, self.last_error())
        return st

    def solve(self, x, w, allow=(OK, ERR_NOT_CONVERGED)):
        """x (n), w (q): FP64 output buffers in the problem's memory kind."""
        R = GqpResult(x=_ptr(x), w=_ptr(w))
        st = self._lib.svm_gqp_solve(self.h, C.byref(R))
        self._check(st, allow)
        out = {k: getattr(R, k) for k, _ in GqpResult._fields_ if k not in ("x", "w", "reserved0")}
        out["status"] = st
        return out

    def project(self, w, x, J=None):
        lam, p = C.c_double(0.0), C.c_int64(0)
        self._check(self._lib.svm_gqp_op_project(self.h, _ptr(w), _ptr(x), C.byref(lam), _ptr(J), C.byref(p)))
        return lam.value, p.value

    def newton(self, J, p, sigma, g, dv):
        self._check(self._lib.svm_gqp_op_newton(self.h, _ptr(J), int(p), float(sigma), _ptr(g), _ptr(dv)))

    def matvec(self, v, z):
        self._check(self._lib.svm_gqp_op_matvec(self.h, _ptr(v), _ptr(z)))

    def rmatvec(self, y, out):
        self._check(self._lib.svm_gqp_op_rmatvec(self.h, _ptr(y), _ptr(out)))
