"""GPU parity of the CSR layout: the products, the Newton direction, the KKT
residual and whole solves through the C ABI, against the FP64 oracle run on
the same matrix stored densely (small cases), and against the KKT residual
recomputed on the host from the sparse matrix (the c3-shaped case, too large
to densify).

Tolerances as for the dense FP64 form: products to 1e-12 of the absolute-sum
scale; the Newton direction to Algorithm 3's CG bound |M dv + g| <=
min(eta, |g|^(1+tau), 1e-10 |g|) (the Jacobi-preconditioned CG's own stop);
solves to relative objective 1e-6 and R_KKT <= 1e-6.
"""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

import paper_1910_01312_gb300 as P  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def make_csr(ip, ix, v, y, q, C=1.0, host_mem=False, **kw):
    if host_mem:
        return P.Solver(None, y, C_=C, csr=(ip, ix, v, q), **kw), None
    keep = (dev(ip), dev(ix), dev(v), dev(y))
    s = P.Solver(None, keep[3], C_=C, csr=(keep[0], keep[1], keep[2], q), **kw)
    return s, keep


def dense(ip, ix, v, q):
    n = ip.size - 1
    return sp.csr_matrix((v, ix, ip), shape=(n, q)).toarray()


def _case(kind, dtype):
    if kind == "zipf":
        ip, ix, v, y, C = datagen.sparse_text(1, n=4001, q=500, nnz_row=30, dtype=dtype)
    elif kind == "text":
        ip, ix, v, y, C = datagen.sparse_text(2, n=20000, q=5000, nnz_row=75, dtype=dtype)
    else:
        # empty rows, empty columns, one column in every row (a column longer than one task)
        rng = np.random.default_rng(3)
        n, q = 6000, 40
        M = np.where(rng.random((n, q)) < 0.1, rng.normal(size=(n, q)), 0.0)
        M[:, 7] = rng.uniform(0.5, 1.0, n)
        M[:, 20:23] = 0.0
        M[100:140] = 0.0
        S = sp.csr_matrix(M)
        S.sort_indices()
        ip, ix, v = S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(dtype)
        y = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
        C = 1.0
    return ip, ix, v, y, C


@pytest.mark.parametrize("prec", [P.PREC_PLAIN_FP64, P.PREC_MIXED])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["zipf", "text", "edges"])
def test_csr_matvec_rmatvec(kind, dtype, prec):
    """PLAIN_FP64: FP64 products.  MIXED with FP32 values: Dot2 in FP32
    (~2^-48 of the absolute sum), within the same 1e-12 bound."""
    ip, ix, v, y, C = _case(kind, dtype)
    n, q = ip.size - 1, {"zipf": 500, "text": 5000, "edges": 40}[kind]
    s, keep = make_csr(ip, ix, v, y, q, C=C, precision=prec)
    X = dense(ip, ix, v, q)
    rng = np.random.default_rng(4)
    w = rng.normal(size=q)
    c = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0, 1, n))
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    o = torch.empty(q, dtype=torch.float64, device="cuda")
    s.matvec(dev(w), z)
    s.rmatvec(dev(c), o)
    zr = oracle.matvec(X, y, w)
    orr, sc = oracle.rmatvec(X, y, c, with_scale=True)
    scale_z = np.abs(X) @ np.abs(w)
    np.testing.assert_array_less(np.abs(host(z) - zr), 1e-12 * scale_z + 1e-300)
    np.testing.assert_array_less(np.abs(host(o) - orr), 1e-12 * sc + 1e-300)
    s.close()


@pytest.mark.parametrize("prec", [P.PREC_PLAIN_FP64, P.PREC_MIXED])
@pytest.mark.parametrize("frac,sigma,gscale", [(0.05, 3.7, 1.0), (0.5, 60.0, 1e-3), (0.002, 1.0, 10.0)])
def test_csr_newton_direction(frac, sigma, gscale, prec):
    """The CG's stop bounds its recurrence residual; the true residual adds the
    products' rounding, 2^-53 (FP64) or ~2^-48 (Dot2) of |M| |dv| per entry."""
    ip, ix, v, y, C = _case("zipf", np.float32 if prec == P.PREC_MIXED else np.float64)
    n, q = ip.size - 1, 500
    X = dense(ip, ix, v, q).astype(np.float64)   # the reference M in FP64 (exact FP32 values)
    rng = np.random.default_rng(5)
    J = np.sort(rng.choice(n, size=max(1, int(frac * n)), replace=False))
    g = gscale * rng.normal(size=q)
    s, keep = make_csr(ip, ix, v, y, q, precision=prec)
    dv = torch.empty(q, dtype=torch.float64, device="cuda")
    s.newton(dev(J.astype(np.int32)), J.size, sigma, dev(g), dv)
    XJ = X[J]
    h = XJ.sum(axis=0)
    M = np.eye(q) + sigma * (XJ.T @ XJ - np.outer(h, h) / J.size)
    gn = np.linalg.norm(g)
    r = np.linalg.norm(M @ host(dv) + g)
    tol = min(0.1, gn ** 1.5, 1e-10 * gn)
    assert r <= 1.001 * tol + 4e-14 * gn * np.linalg.norm(M, 2), (r, tol)
    dv_r = oracle.newton_direction(X, y, J.astype(np.int64), sigma, g, form=1)
    np.testing.assert_allclose(host(dv), dv_r, rtol=0, atol=1e-8 * np.linalg.norm(dv_r))
    s.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_csr_kkt_residual(dtype):
    ip, ix, v, y, C = _case("zipf", dtype)
    q = 500
    X = dense(ip, ix, v, q)
    a, _ = oracle.project(np.random.default_rng(6).uniform(0, C, y.size), y, C)
    s, keep = make_csr(ip, ix, v, y, q, C=C)
    r, lam = s.kkt(dev(a))
    assert r == pytest.approx(oracle.kkt(X, y, C, a), rel=1e-9)
    s.close()


def _solve(s, n, q, alpha0=None):
    alpha = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(q, dtype=torch.float64, device="cuda")
    r = s.solve(alpha, w, alpha0=alpha0)
    return r, host(alpha), host(w)


@pytest.mark.parametrize("dtype,C", [(np.float32, 1.0), (np.float64, 0.2), (np.float32, 20.0)])
def test_csr_solve_matches_oracle(dtype, C):
    ip, ix, v, y, _ = datagen.sparse_text(7, n=3000, q=400, nnz_row=30, dtype=dtype)
    q = 400
    X = dense(ip, ix, v, q)
    ref = oracle.solve(X, y, C, tol=1e-10)
    s, keep = make_csr(ip, ix, v, y, q, C=C)
    r, alpha, w = _solve(s, y.size, q)
    assert r["status"] == P.OK and r["kkt"] <= 1e-6, r
    assert oracle.kkt(X, y, C, alpha) <= 1e-6
    assert alpha.min() >= 0.0 and alpha.max() <= C
    assert r["objective"] == pytest.approx(ref["objective"], rel=1e-6)
    # f(alpha) - f* >= |A'alpha - A'alpha*|^2 / 2 for feasible alpha (f is quadratic
    # with Hessian AA' and alpha* satisfies the first-order condition), so the
    # objective gap bounds w's error
    dfo = max(r["objective"] - ref["objective"], 1e-13 * abs(ref["objective"]))
    assert np.linalg.norm(w - ref["w"]) <= 1.01 * np.sqrt(2.0 * dfo) + 1e-9 * np.linalg.norm(ref["w"])
    # the same problem through the dense FP64 form reaches the same optimum
    sd = P.Solver(dev(X), dev(y), C_=C, precision=P.PREC_PLAIN_FP64)
    rd, ad, wd = _solve(sd, y.size, q)
    assert r["objective"] == pytest.approx(rd["objective"], rel=1e-8)
    s.close()
    sd.close()


def test_csr_host_memory_and_warm_start():
    ip, ix, v, y, C = datagen.sparse_text(8, n=2500, q=300, nnz_row=25)
    q = 300
    X = dense(ip, ix, v, q)
    ref = oracle.solve(X, y, C, tol=1e-10)
    s, _ = make_csr(ip, ix, v, y, q, C=C, host_mem=True)
    alpha, w = np.zeros(y.size), np.zeros(q)
    r = s.solve(alpha, w)
    assert r["status"] == P.OK and r["objective"] == pytest.approx(ref["objective"], rel=1e-6)
    r2 = s.solve(alpha.copy(), w, alpha0=alpha.copy())
    assert r2["status"] == P.OK and r2["outer_iters"] <= 2
    s.close()


def test_csr_invalid_structure():
    ip = np.array([0, 2, 3], np.int64)
    y = np.array([1, -1], np.int8)
    v = np.ones(3, np.float32)
    for ix, q in [(np.array([1, 0, 0], np.int32), 4),     # columns not increasing
                  (np.array([0, 0, 1], np.int32), 4),     # repeated column
                  (np.array([0, 5, 1], np.int32), 4)]:    # column out of range
        with pytest.raises(P.SVMError) as e:
            make_csr(ip, ix, v, y, q)
        assert e.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.SVMError) as e:
        make_csr(np.array([0, 2, 4], np.int64), np.array([0, 1, 2], np.int32), v, y, 4)   # indptr[n] != nnz
    assert e.value.status == P.ERR_INVALID_ARG


def test_csr_text_shaped_solve():
    """The c3 recipe at n = 10^5 (q = 47,000, 75 entries per row): too large to
    densify, so R_KKT of the returned alpha is recomputed on the host from the
    sparse matrix (scipy products, the oracle's projection)."""
    ip, ix, v, y, C = datagen.sparse_text(0, n=100_000)
    q = 47_000
    s, keep = make_csr(ip, ix, v, y, q, C=C)
    r, alpha, w = _solve(s, y.size, q)
    assert r["status"] == P.OK and r["kkt"] <= 1e-6, r
    X = sp.csr_matrix((v.astype(np.float64), ix, ip), shape=(y.size, q))
    yf = y.astype(np.float64)
    wr = X.T @ (yf * alpha)
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-9 * max(1.0, np.abs(wr).max()))
    grad = yf * (X @ wr) - 1.0
    pi, _ = oracle.project(alpha - grad, y, C)
    R = np.linalg.norm(alpha - pi) / (1.0 + np.linalg.norm(alpha))
    # the solver's own target; 1e-9 covers the rounding between two FP64 evaluations
    assert R <= 1e-6 + 1e-9, (R, r["kkt"])
    assert r["objective"] == pytest.approx(0.5 * wr @ wr - alpha.sum(), rel=1e-9)
    s.close()
