"""GPU parity of the unified-QP solver (eq. (1.5)) and of the SVR dual (eqs.
(1.3)-(1.4)) through the C ABI (include/svm_gqp.h), against the FP64
reference oracle/gqp.py (itself pinned in test_gqp_oracle.py by projection
patterns, the C-SVC oracle, active-set enumeration and the SVR's zero gap).

The GPU path is FP64 throughout, so steps agree with the reference to a few
ulps of the summed magnitudes (1e-12 of the absolute-sum scale), index sets
exactly except for components within roundoff of a bound, and whole solves on
what is unique: the objective (relative 1e-6), both sides' R_KKT <= 1e-6,
feasibility and, for the SVR, the zero primal-dual gap.  The references are
solved to R_KKT <= 1e-9 (general QPs) and 1e-8 (SVR duals): tighter targets
are below the FP64 reference's own roundoff floor on some of these problems
(it then spends its 200 outer iterations raising sigma), and these already
fix the objective far inside the 1e-6 being checked.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle import gqp

torch = pytest.importorskip("torch")
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
    return t.detach().cpu().numpy()


def _general_problem(rng, n, q, dtype=np.float64, zeros=True):
    """Signed, non-unit a with a few zeros, per-component boxes l < u (and one
    fixed variable l = u), d != 0 inside the reachable range, any c."""
    B = rng.normal(size=(n, q)).astype(dtype)
    c = rng.normal(size=n)
    a = rng.normal(size=n) * rng.uniform(0.2, 3.0, size=n)
    if zeros:
        a[rng.choice(n, size=max(1, n // 50), replace=False)] = 0.0
    lo = rng.normal(size=n)
    hi = lo + rng.uniform(0.1, 2.0, size=n)
    hi[0] = lo[0]                                   # a fixed variable
    d = float(a @ rng.uniform(lo, hi))
    return B, c, a, d, lo, hi


def _handle(B, c, a, d, lo, hi, stacked=False, **kw):
    keep = [dev(B), dev(c), dev(a), dev(lo), dev(hi)]
    h = P.GQP(*keep, d=d, stacked=stacked, **kw)
    return h, keep


# ------------------------------------------------------------------ products

@pytest.mark.parametrize("stacked", [False, True])
@pytest.mark.parametrize("dtype,m,q", [(np.float64, 1000, 7), (np.float32, 3001, 128), (np.float32, 513, 300),
                                       (np.float64, 1, 1)])
def test_products(stacked, dtype, m, q):
    rng = np.random.default_rng(m + q)
    X = rng.normal(size=(m, q)).astype(dtype)
    n = 2 * m if stacked else m
    Bf = np.vstack([X, -X]).astype(np.float64) if stacked else X.astype(np.float64)
    ones = np.ones(n)
    h, keep = _handle(X, ones, ones, 0.0, -ones * 10, ones * 10, stacked=stacked)
    v = rng.normal(size=q)
    y = np.where(rng.random(n) < 0.3, 0.0, rng.normal(size=n))
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    o = torch.empty(q, dtype=torch.float64, device="cuda")
    h.matvec(dev(v), z)
    h.rmatvec(dev(y), o)
    np.testing.assert_array_less(np.abs(host(z) - Bf @ v), 1e-12 * (np.abs(Bf) @ np.abs(v)) + 1e-300)
    np.testing.assert_array_less(np.abs(host(o) - Bf.T @ y), 1e-12 * (np.abs(Bf).T @ np.abs(y)) + 1e-300)
    h.close()


# ---------------------------------------------------------------- projection

@pytest.mark.parametrize("n", [1, 7, 1000, 50_001])
def test_projection_general_a(n):
    rng = np.random.default_rng(n)
    _, c, a, d, lo, hi = _general_problem(rng, n, 1, zeros=n > 1)
    if n == 1:
        a[0] = 1.5
        lo[0], hi[0] = -1.0, 2.0
        d = 0.75
    h, keep = _handle(np.zeros((n, 1)), c, a, d, lo, hi)
    for trial in range(3):
        w = rng.normal(size=n) * 3.0
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        J = torch.empty(n, dtype=torch.int32, device="cuda")
        lam, p = h.project(dev(w), x, J)
        xr, lam_r = gqp.project(w, a, d, lo, hi)
        scale = np.max(np.abs(w)) + np.max(np.abs(hi)) + np.max(np.abs(lo))
        xg = host(x)
        np.testing.assert_allclose(xg, xr, rtol=0, atol=1e-12 * scale)
        assert np.all(xg >= lo) and np.all(xg <= hi)
        assert abs(a @ xg - d) <= 1e-11 * (1 + np.abs(a) @ np.abs(xg))
        r = w - lam * a
        np.testing.assert_array_equal(xg, np.clip(r, lo, hi))      # x = clip(w - lambda a) exactly
        Jr = gqp.free_set(w, a, lo, hi, lam_r)
        Jg = host(J)[:p]
        amb = np.minimum(np.abs(r - lo), np.abs(r - hi)) <= 1e-11 * scale
        assert all(amb[i] for i in set(Jg.tolist()) ^ set(Jr.tolist()))
        assert list(Jg) == sorted(Jg)
    h.close()


def test_projection_worked_example_and_ties():
    """Worked by hand: w = (1, 2, 0.5, -1), a = (1, -1, 0, 2), l = (0, 0, 0, -3),
    u = (1, 3, 1, 0), d = -0.5; x(lambda) = clip(w - lambda a, l, u).
    At lambda = 0: x = (1, 2, 0.5, -1), a'x = -3 < d, and a'x(lambda) falls
    as lambda grows, so the root is negative.  For -0.5 <= lambda <= 0:
    x1 = 1 (at u), x2 = 2 + lambda, x3 = 0.5 (a = 0), x4 = -1 - 2 lambda, so
    a'x = 1 - (2 + lambda) + 2 (-1 - 2 lambda) = -3 - 5 lambda = -0.5 at
    lambda = -0.5 (left of it the slope is -1: the root is unique).  Then
    x = (1, 1.5, 0.5, 0) with x4 exactly at its upper bound (a tie: active),
    and J = {1, 2} (x3 is strictly inside its box although a_3 = 0)."""
    w = np.array([1.0, 2.0, 0.5, -1.0])
    a = np.array([1.0, -1.0, 0.0, 2.0])
    lo = np.array([0.0, 0.0, 0.0, -3.0])
    hi = np.array([1.0, 3.0, 1.0, 0.0])
    h, keep = _handle(np.zeros((4, 1)), np.zeros(4), a, -0.5, lo, hi)
    x = torch.empty(4, dtype=torch.float64, device="cuda")
    J = torch.empty(4, dtype=torch.int32, device="cuda")
    lam, p = h.project(dev(w), x, J)
    assert lam == pytest.approx(-0.5, abs=1e-15)
    np.testing.assert_allclose(host(x), [1.0, 1.5, 0.5, 0.0], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(host(J)[:p], [1, 2])
    h.close()


# ---------------------------------------------------------------- Newton

@pytest.mark.parametrize("stacked", [False, True])
@pytest.mark.parametrize("m,q,frac", [(400, 12, 0.3), (3000, 64, 0.05), (600, 150, 0.5)])
def test_newton_direction(stacked, m, q, frac):
    rng = np.random.default_rng(q)
    X = rng.normal(size=(m, q))
    n = 2 * m if stacked else m
    Bf = np.vstack([X, -X]) if stacked else X
    a = rng.normal(size=n)
    a[::17] = 0.0
    h, keep = _handle(X, np.zeros(n), a, 0.0, -np.ones(n) * 1e3, np.ones(n) * 1e3, stacked=stacked)
    J = np.sort(rng.choice(n, size=max(1, int(frac * n)), replace=False)).astype(np.int32)
    g = rng.normal(size=q)
    for sigma in (1.0, 125.0):
        dv = torch.empty(q, dtype=torch.float64, device="cuda")
        h.newton(dev(J), J.size, sigma, dev(g), dv)
        ref = gqp.newton_direction(Bf, a, J.astype(np.int64), sigma, g)
        M = np.eye(q) + sigma * Bf[J].T @ Bf[J]
        cond = np.linalg.cond(M)
        np.testing.assert_allclose(host(dv), ref, rtol=0, atol=1e-13 * cond * (1 + np.abs(ref).max()))
    # no free rows: case (b) of Prop. 3.5, dv = -g
    dv = torch.empty(q, dtype=torch.float64, device="cuda")
    h.newton(None, 0, 1.0, dev(g), dv)
    np.testing.assert_array_equal(host(dv), -g)
    h.close()


def test_newton_all_free_a_zero_has_no_rank_one_term():
    """a_J = 0 on the free set: the HS-Jacobian has no rank-one part (s = 0)."""
    rng = np.random.default_rng(3)
    B = rng.normal(size=(50, 6))
    a = np.zeros(50)
    a[0] = 1.0
    h, keep = _handle(B, np.zeros(50), a, 0.0, -np.ones(50), np.ones(50))
    J = np.arange(1, 50, dtype=np.int32)
    g = rng.normal(size=6)
    dv = torch.empty(6, dtype=torch.float64, device="cuda")
    h.newton(dev(J), J.size, 2.0, dev(g), dv)
    ref = np.linalg.solve(np.eye(6) + 2.0 * B[1:].T @ B[1:], -g)
    np.testing.assert_allclose(host(dv), ref, rtol=1e-12, atol=1e-13)
    h.close()


# ---------------------------------------------------------------- whole solves

def _check_solve(r, x, w, B, c, a, d, lo, hi, ref):
    assert r["status"] == P.OK, r
    assert r["kkt"] <= 1e-6
    assert gqp.kkt(B, c, a, d, lo, hi, x) <= 1e-6
    assert np.all(x >= lo) and np.all(x <= hi)
    assert abs(a @ x - d) <= 1e-9 * (1 + np.abs(a) @ np.abs(x))
    assert r["feasibility"] == pytest.approx(a @ x - d, abs=1e-9 * (1 + np.abs(a) @ np.abs(x)))
    np.testing.assert_allclose(w, B.T @ x, rtol=0, atol=1e-10 * (1 + np.abs(B).T @ np.abs(x)).max())
    assert r["objective"] == pytest.approx(ref["objective"], rel=1e-6, abs=1e-9)
    assert r["objective"] == pytest.approx(gqp.objective(B, c, x), rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("n,q,seed,dtype", [(300, 5, 0, np.float64), (2000, 40, 1, np.float32),
                                            (1500, 200, 2, np.float64), (40, 3, 3, np.float64)])
def test_solve_general_qp(n, q, seed, dtype):
    rng = np.random.default_rng(seed)
    B, c, a, d, lo, hi = _general_problem(rng, n, q, dtype)
    ref = gqp.solve(B.astype(np.float64), c, a, d, lo, hi, tol=1e-9)
    assert ref["status"] == "ok"
    h, keep = _handle(B, c, a, d, lo, hi, tol=1e-6)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    w = torch.empty(q, dtype=torch.float64, device="cuda")
    r = h.solve(x, w)
    _check_solve(r, host(x), host(w), B.astype(np.float64), c, a, d, lo, hi, ref)
    h.close()


def test_solve_host_memory():
    rng = np.random.default_rng(9)
    B, c, a, d, lo, hi = _general_problem(rng, 500, 8)
    ref = gqp.solve(B, c, a, d, lo, hi, tol=1e-9)
    h = P.GQP(B, c, a, lo, hi, d=d, tol=1e-6)
    x, w = np.zeros(500), np.zeros(8)
    r = h.solve(x, w)
    _check_solve(r, x, w, B, c, a, d, lo, hi, ref)
    h.close()


def test_tiny_qp_against_active_set_enumeration():
    """n = 6: the reference's own pin (enumeration of the QP's faces) checked
    directly against the GPU's objective."""
    import importlib
    pins = importlib.import_module("test_gqp_oracle")
    rng = np.random.default_rng(21)
    for trial in range(3):
        B = rng.normal(size=(6, 3))
        c = rng.normal(size=6)
        a, d, lo, hi = pins._box_problem(rng, 6)
        best = pins._qp_by_active_sets(B, c, a, d, lo, hi)
        h, keep = _handle(B, c, a, d, lo, hi, tol=1e-9)
        x = torch.empty(6, dtype=torch.float64, device="cuda")
        w = torch.empty(3, dtype=torch.float64, device="cuda")
        r = h.solve(x, w)
        assert r["status"] == P.OK
        assert abs(r["objective"] - best) <= 1e-7 * (1 + abs(best)), (trial, r["objective"], best)
        h.close()


def test_csvc_as_unified_qp_matches_the_c_oracle():
    X, y = datagen.small(2000, 30, seed=4)
    C = 0.5
    yf = y.astype(np.float64)
    n = X.shape[0]
    ref = oracle.solve(X, y, C, tol=1e-10)
    h, keep = _handle(X * yf[:, None], -np.ones(n), yf, 0.0, np.zeros(n), np.full(n, C))
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    w = torch.empty(30, dtype=torch.float64, device="cuda")
    r = h.solve(x, w)
    assert r["status"] == P.OK and r["kkt"] <= 1e-6
    assert oracle.kkt(X, y, C, host(x)) <= 1e-6
    assert r["objective"] == pytest.approx(ref["objective"], rel=1e-6)
    assert r["lam"] == pytest.approx(ref["lam_kkt"], abs=1e-4)      # the C-SVC's bias b
    h.close()


def test_infeasible_and_invalid_problems_are_rejected():
    n = 5
    a = np.ones(n)
    with pytest.raises(P.SVMError) as e:           # a'x <= 5 < d = 7 on the box [0, 1]^5
        _handle(np.ones((n, 2)), np.zeros(n), a, 7.0, np.zeros(n), np.ones(n))
    assert e.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.SVMError) as e:           # l > u
        _handle(np.ones((n, 2)), np.zeros(n), a, 0.0, np.ones(n), np.zeros(n))
    assert e.value.status == P.ERR_INVALID_ARG
    c = np.zeros(n)
    c[2] = np.nan
    with pytest.raises(P.SVMError) as e:
        _handle(np.ones((n, 2)), c, a, 0.0, np.zeros(n), np.ones(n))
    assert e.value.status == P.ERR_INVALID_ARG


# ---------------------------------------------------------------- SVR

@pytest.mark.parametrize("m,q,eps,C,dtype", [(600, 4, 0.1, 1.0, np.float64), (2000, 20, 0.05, 10.0, np.float32),
                                             (300, 50, 0.5, 0.1, np.float64)])
def test_svr_matches_reference_with_zero_gap(m, q, eps, C, dtype):
    """eq. (1.4) at Tol 1e-6 (the paper's SVR tolerance, Sec. 4.4): the GPU
    dual's objective against the reference's, and the primal of eq. (1.3) at
    the returned w_svr = X'(z - x), b = -lambda: equal (up to the tolerance) to
    minus the dual objective, and to the primal minimised over b."""
    rng = np.random.default_rng(m)
    X = rng.normal(size=(m, q)).astype(dtype)
    wt = rng.normal(size=q)
    y = X.astype(np.float64) @ wt + 0.3 * rng.normal(size=m)
    Xf = X.astype(np.float64)
    ref = gqp.solve(*gqp.svr_problem(Xf, y, eps, C), tol=1e-8)
    assert ref["status"] == "ok"
    keep = (dev(X), dev(y))
    h = P.GQP.svr(keep[0], keep[1], eps, C, tol=1e-6)
    x = torch.empty(2 * m, dtype=torch.float64, device="cuda")
    w = torch.empty(q, dtype=torch.float64, device="cuda")
    r = h.solve(x, w)
    assert r["status"] == P.OK and r["kkt"] <= 1e-6
    xg = host(x)
    B, c, a, d, lo, hi = gqp.svr_problem(Xf, y, eps, C)
    assert gqp.kkt(B, c, a, d, lo, hi, xg) <= 1e-6
    assert r["objective"] == pytest.approx(ref["objective"], rel=1e-6)
    beta = xg[m:] - xg[:m]
    w_svr = -host(w)
    np.testing.assert_allclose(w_svr, Xf.T @ beta, rtol=0, atol=1e-9 * (1 + np.abs(Xf).T @ np.abs(beta)).max())
    b = -r["lam"]
    resid = y - Xf @ w_svr
    primal_b = 0.5 * w_svr @ w_svr + C * np.maximum(0.0, np.abs(resid - b) - eps).sum()
    primal_min, _ = gqp.svr_primal(Xf, y, eps, C, w_svr)
    dual = -r["objective"]
    scale = abs(primal_min) + 1.0
    assert primal_min - dual >= -1e-8 * scale                 # weak duality
    assert primal_min - dual <= 2e-5 * scale                  # no gap, up to the solve's tolerance
    assert primal_b - primal_min <= 2e-5 * scale              # b = -lambda minimises the primal in b
    h.close()
