"""Pins of the unified-QP reference (oracle/gqp.py, eq. (1.5)) against
results fixed independently of its own code: the optimality patterns of the
projection, the C-SVC oracle (itself pinned by brute force), an enumeration
of a tiny QP's active sets, and the zero primal-dual gap of the SVR."""
import itertools

import numpy as np

import datagen
import oracle
from oracle import gqp


def _box_problem(rng, n):
    a = rng.normal(size=n) * rng.uniform(0.2, 3.0, size=n)
    a[rng.integers(n)] = 0.0                      # a component the constraint does not see
    lo = rng.normal(size=n)
    hi = lo + rng.uniform(0.1, 2.0, size=n)
    x0 = rng.uniform(lo, hi)
    return a, float(a @ x0), lo, hi


def _projection_by_patterns(u, a, d, lo, hi):
    """The unique point x = clip(u - lam a, lo, hi) with a'x = d, found by trying
    every assignment of the components to {lower, upper, free}."""
    n = u.size
    found = []
    for pat in itertools.product((0, 1, 2), repeat=n):
        pat = np.array(pat)
        L, U, F = pat == 0, pat == 1, pat == 2
        s = float(a[F] @ a[F])
        if s == 0.0:
            continue
        lam = (a[F] @ u[F] + a[L] @ lo[L] + a[U] @ hi[U] - d) / s
        r = u - lam * a
        ok = np.all(r[F] >= lo[F] - 1e-12) and np.all(r[F] <= hi[F] + 1e-12) \
            and np.all(r[L] <= lo[L] + 1e-12) and np.all(r[U] >= hi[U] - 1e-12)
        if ok:
            found.append(np.clip(r, lo, hi))
    assert found
    return found[0], found


def test_projection_against_pattern_enumeration():
    rng = np.random.default_rng(0)
    for trial in range(25):
        n = 6
        a, d, lo, hi = _box_problem(rng, n)
        u = rng.normal(size=n) * 2.0
        x, lam = gqp.project(u, a, d, lo, hi)
        xr, allx = _projection_by_patterns(u, a, d, lo, hi)
        for xx in allx:                            # every consistent pattern gives the same point
            np.testing.assert_allclose(xx, xr, rtol=0, atol=1e-10)
        np.testing.assert_allclose(x, xr, rtol=0, atol=1e-10)
        assert abs(a @ x - d) <= 1e-10 * (1 + np.abs(a) @ np.abs(x))
        assert np.all(x >= lo) and np.all(x <= hi)


def test_csvc_case_matches_the_c_oracle():
    X, y = datagen.small(80, 5, seed=3)
    C = 1.0
    yf = y.astype(np.float64)
    n = X.shape[0]
    r = gqp.solve(X * yf[:, None], -np.ones(n), yf, 0.0, np.zeros(n), np.full(n, C), tol=1e-10)
    ref = oracle.solve(X, y, C, tol=1e-10)
    assert r["status"] == "ok" and r["kkt"] <= 1e-10
    assert abs(r["objective"] - ref["objective"]) <= 1e-9 * abs(ref["objective"])


def _qp_by_active_sets(B, c, a, d, lo, hi):
    """min over the faces {x_i at l_i, at u_i or free}: on each face the
    equality-constrained QP's KKT system (minimum-norm least squares, Q may be
    singular); the smallest objective among the feasible stationary points."""
    n = c.size
    Q = B @ B.T
    best = np.inf
    for pat in itertools.product((0, 1, 2), repeat=n):
        pat = np.array(pat)
        F = np.nonzero(pat == 2)[0]
        N = np.nonzero(pat != 2)[0]
        xN = np.where(pat[N] == 0, lo[N], hi[N])
        x = np.zeros(n)
        x[N] = xN
        if F.size == 0:
            if abs(a[N] @ xN - d) > 1e-10:
                continue
        else:
            K = np.zeros((F.size + 1, F.size + 1))
            K[:F.size, :F.size] = Q[np.ix_(F, F)]
            K[:F.size, F.size] = a[F]
            K[F.size, :F.size] = a[F]
            rhs = np.concatenate([-(c[F] + Q[np.ix_(F, N)] @ xN), [d - a[N] @ xN]])
            sol, *_ = np.linalg.lstsq(K, rhs, rcond=None)
            if np.linalg.norm(K @ sol - rhs) > 1e-9 * (1 + np.linalg.norm(rhs)):
                continue
            x[F] = sol[:F.size]
            if np.any(x[F] < lo[F] - 1e-10) or np.any(x[F] > hi[F] + 1e-10):
                continue
        best = min(best, 0.5 * x @ Q @ x + c @ x)
    return best


def test_tiny_qps_against_active_set_enumeration():
    rng = np.random.default_rng(7)
    for trial in range(6):
        n, q = 6, 3
        B = rng.normal(size=(n, q))
        c = rng.normal(size=n)
        a, d, lo, hi = _box_problem(rng, n)
        r = gqp.solve(B, c, a, d, lo, hi, tol=1e-11)
        ref = _qp_by_active_sets(B, c, a, d, lo, hi)
        assert r["status"] == "ok"
        assert abs(r["objective"] - ref) <= 1e-8 * (1 + abs(ref)), (trial, r["objective"], ref)


def test_svr_dual_has_zero_gap_with_the_svr_primal():
    # eq. (1.4) with the linear kernel: the minimum of the dual is minus the primal
    # optimum 1/2 |w|^2 + C sum max(0, |y - w'x - b| - eps), w = X'(z - x)
    rng = np.random.default_rng(11)
    n, q, eps, C = 40, 3, 0.1, 1.0
    X = rng.normal(size=(n, q))
    y = X @ np.array([1.0, -2.0, 0.5]) + 0.3 * rng.normal(size=n)
    r = gqp.solve(*gqp.svr_problem(X, y, eps, C), tol=1e-11)
    assert r["status"] == "ok"
    xx, zz = r["x"][:n], r["x"][n:]
    assert abs(xx.sum() - zz.sum()) <= 1e-9 * (1 + xx.sum())
    w = X.T @ (zz - xx)
    primal, b = gqp.svr_primal(X, y, eps, C, w)
    assert primal + r["objective"] >= -1e-9 * abs(primal)          # weak duality
    assert primal + r["objective"] <= 1e-8 * abs(primal)           # and no gap at the optimum


def test_free_set_sends_ties_to_the_bound():
    # components exactly at a bound after the shift are active (the paper's clip sends
    # t >= u to u and t <= l to l), so J holds strict interior points only
    u = np.array([1.0, 2.0, 0.5, -1.0])
    a = np.array([1.0, -1.0, 0.0, 2.0])
    lo = np.array([0.0, 0.0, 0.0, -3.0])
    hi = np.array([1.0, 3.0, 1.0, 0.0])
    lam = 1.0          # r = u - lam a = [0, 3, 0.5, -3]: lower tie, upper tie, interior, lower tie
    np.testing.assert_array_equal(gqp.free_set(u, a, lo, hi, lam), [2])
