"""Pins of the oracle's CSR loops (the sparse workload's products and R_KKT).

A CSR row holds the nonzero entries of the dense row in column order, and the
dense loops only add zero terms besides them, so the CSR products must equal
the dense oracle's on the densified matrix bit for bit (the dense oracle is
pinned in test_oracle_pins.py); scipy's sparse products are a second,
independent check, and the hand-worked R_KKT examples pin kkt_csr directly.
"""
import os

import numpy as np
import pytest

import datagen
import oracle

sp = pytest.importorskip("scipy.sparse")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(ip, ix, v, q):
    X = np.zeros((ip.size - 1, q), dtype=v.dtype)
    for i in range(ip.size - 1):
        X[i, ix[ip[i]:ip[i + 1]]] = v[ip[i]:ip[i + 1]]
    return X


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,q,nnz_row,seed", [(300, 50, 7, 0), (2000, 400, 30, 1), (77, 5, 3, 2)])
def test_csr_products_equal_dense_oracle(dtype, n, q, nnz_row, seed):
    ip, ix, v, y, _ = datagen.sparse_text(seed, n=n, q=q, nnz_row=nnz_row, dtype=dtype)
    X = _dense(ip, ix, v, q)
    rng = np.random.default_rng(seed)
    w = rng.normal(size=q)
    c = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0, 1, n))
    z = oracle.matvec_csr(ip, ix, v, q, y, w)
    o = oracle.rmatvec_csr(ip, ix, v, q, y, c)
    np.testing.assert_array_equal(z, oracle.matvec(X, y, w))
    np.testing.assert_array_equal(o, oracle.rmatvec(X, y, c))
    S = sp.csr_matrix((v.astype(np.float64), ix, ip), shape=(n, q))
    yf = y.astype(np.float64)
    absz = abs(S) @ np.abs(w)
    np.testing.assert_array_less(np.abs(z - yf * (S @ w)), 1e-14 * absz + 1e-300)
    abso = abs(S).T @ np.abs(c)
    np.testing.assert_array_less(np.abs(o - S.T @ (yf * c)), 1e-14 * abso + 1e-300)


@pytest.mark.parametrize("C", [0.05, 1.0])
def test_csr_kkt_equals_dense_oracle(C):
    ip, ix, v, y, _ = datagen.sparse_text(3, n=1500, q=200, nnz_row=20)
    X = _dense(ip, ix, v, 200)
    a = np.random.default_rng(4).uniform(0, C, y.size)
    r1, l1, w1 = oracle.kkt_csr(ip, ix, v, 200, y, C, a, with_extras=True)
    r2, l2, w2 = oracle.kkt(X, y, C, a, with_extras=True)
    assert r1 == r2 and l1 == l2
    np.testing.assert_array_equal(w1, w2)
    r3 = oracle.kkt_csr(ip, ix, v, 200, y, C, a, omp=True)
    assert r3 == r1


@pytest.mark.parametrize("ex", ["1", "2"])
def test_csr_kkt_hand_worked_examples(ex):
    g = {}
    for line in open(os.path.join(GOLDEN, "kkt_worked.txt")):
        if line.strip() and not line.startswith("#"):
            k, *vals = line.split()
            g[k] = np.array([float(x) for x in vals])
    y = g["y" + ex].astype(np.int8)
    X = g["X" + ex].reshape(y.size, -1)
    S = sp.csr_matrix(X)
    r, lam, _ = oracle.kkt_csr(S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data, X.shape[1], y,
                               g["C" + ex][0], g["alpha" + ex], with_extras=True)
    assert r == pytest.approx(g["R" + ex][0], rel=1e-14)
    assert lam == pytest.approx(g["lambda" + ex][0], abs=1e-14)


def test_openmp_build_is_bit_identical():
    """The all-core build used for the CPU baseline computes the same solve."""
    X, y, C = datagen.gauss1m(1, n=40_000)
    a = oracle.solve(X, y, C, tol=1e-6)
    b = oracle.solve(X, y, C, tol=1e-6, omp=True)
    np.testing.assert_array_equal(a["alpha"], b["alpha"])
    np.testing.assert_array_equal(a["w"], b["w"])
    assert a["objective"] == b["objective"] and a["kkt"] == b["kkt"]
    assert (a["outer"], a["inner_total"]) == (b["outer"], b["inner_total"])
