"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that the headers under include/ declare (no GPU
calls)."""
import glob
import os
import re
import subprocess

import pytest

import paper_1910_01312_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(svm_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported():
    lib = P.build()
    P.load()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert set(P.SYMBOLS) == set(declared)


def test_default_params():
    p = P.default_params()
    assert p.tol == 1e-6 and p.max_outer == 200 and p.sigma0 == 1.0
    assert p.precision == P.PREC_MIXED


def test_create_rejects_bad_args_without_gpu_work():
    import numpy as np
    X = np.zeros((4, 3))
    y = np.array([1, -1, 1, -1], np.int8)
    with pytest.raises(P.SVMError) as e:
        P.Solver(X, y, C_=-1.0)
    assert e.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.SVMError) as e:
        P.Solver(X, y, C_=float("nan"))
    assert e.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.SVMError) as e:
        P.Solver(np.zeros((4, 2000), np.float32), y, C_=1.0)
    assert e.value.status == P.ERR_UNSUPPORTED


def test_entry_points_reject_bad_arguments_before_any_gpu_work():
    """Argument checks come before any CUDA call, so they hold without a GPU."""
    import numpy as np
    L = P.load()
    buf = np.zeros(64, np.float32)
    p = buf.ctypes.data
    # random features: null pointers and empty sizes, then an unaligned output
    assert L.svm_rff_features(None, 4, 3, p, 2, p, None) == P.ERR_INVALID_ARG
    assert L.svm_rff_features(p, 0, 3, p, 2, p, None) == P.ERR_INVALID_ARG
    assert L.svm_rff_features(p, 4, 3, p, 0, p, None) == P.ERR_INVALID_ARG
    assert L.svm_rff_features(p, 4, 3, p, 2, p + 4, None) == P.ERR_UNSUPPORTED
    # batched solve and step-level entry points on a null handle
    R = (P.binding.Result * 2)()
    cs = np.ones(2)
    assert L.svm_ssnalm_solve_batch(None, 2, p, cs.ctypes.data, p, p, R) == P.ERR_INVALID_ARG
    assert L.svm_op_gram(None, p, 1, p, p) == P.ERR_INVALID_ARG
    assert L.svm_ssnalm_solve(None, None, None) == P.ERR_INVALID_ARG
    # the allocation-free product: sizes beyond its limit, null pointers
    assert L.svm_rmatvec_noalloc(p, p, 10, 4096, p, p, None) == P.ERR_UNSUPPORTED
    assert L.svm_rmatvec_noalloc(None, p, 10, 4, p, p, None) == P.ERR_INVALID_ARG


def test_binding_rejects_non_contiguous_buffers():
    import numpy as np
    X = np.zeros((6, 4), order="F")
    with pytest.raises(ValueError):
        P.binding._ptr(X)
    assert P.binding._ptr(np.zeros((6, 4))) != 0 and P.binding._ptr(None) is None


def test_noalloc_binding_rejects_wrong_buffers_before_the_call():
    """The allocation-free product trusts its pointers, so the binding checks
    dtypes, shapes and devices first (no GPU needed: the checks raise before
    any C call)."""
    torch = pytest.importorskip("torch")
    n, q = 6, 4
    X = torch.zeros((n, q), dtype=torch.float32)
    y = torch.ones(n, dtype=torch.int8)
    c = torch.zeros(n, dtype=torch.float64)
    out = torch.zeros(q, dtype=torch.float64)
    chk = P.binding._check_noalloc_args
    with pytest.raises(TypeError):
        chk(X.double(), y, c, out)                  # FP64 X
    with pytest.raises(TypeError):
        chk(X, y.to(torch.int32), c, out)            # labels not int8
    with pytest.raises(TypeError):
        chk(X, y, c.float(), out)                    # FP32 weights: the kernel would read 8n bytes
    with pytest.raises(TypeError):
        chk(X, y, c, out.float())                    # FP32 output: the kernel would write 8q bytes
    with pytest.raises(ValueError):
        chk(X, y, c[:-1], out)                       # short c
    with pytest.raises(ValueError):
        chk(X, y, c, torch.zeros(q - 1, dtype=torch.float64))   # short out
    with pytest.raises(ValueError):
        chk(X.reshape(-1), y, c, out)                # X not 2-D
    with pytest.raises(ValueError):
        chk(X, y, c, out)                            # host tensors
    with pytest.raises(TypeError):
        chk(X.numpy(), y, c, out)                    # not a tensor
