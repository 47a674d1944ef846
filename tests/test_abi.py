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
