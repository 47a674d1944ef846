"""Pins that tie the FP64 oracle to the paper and to mathematics, not to itself.

Each test checks an oracle function against something it cannot share a
mistake with: a hand-worked example, a closed form, brute-force enumeration,
finite differences, an independent library routine (numpy's dense algebra) or
an invariant the paper states.  All run on the CPU.
"""
import itertools
import os

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vals = line.split()
            out[k] = np.array([float(v) for v in vals])
    return out


# --------------------------------------------------------------- projection

def test_projection_worked_example():
    """Hand-worked example of Sec. 3.2.1 (Algorithm 2 then the clip)."""
    g = _read_golden("projection_worked_n4.txt")
    y = g["y"].astype(np.int8)
    pi, lam = oracle.project(g["u"], y, g["C"][0])
    assert lam == pytest.approx(g["lambda"][0], abs=1e-15)
    np.testing.assert_allclose(pi, g["pi"], atol=1e-15)
    J = oracle.free_set(g["u"], y, g["C"][0], lam)
    np.testing.assert_array_equal(J, g["J"].astype(np.int64))


def _proj_bruteforce(u, y, C):
    """Projection onto {y'x=0, 0<=x<=C} by enumerating lower/upper/free
    patterns: on the free set x_F = u_F - lam y_F with lam from y'x = 0."""
    n = u.size
    best, bestx = np.inf, None
    for pat in itertools.product((0, 1, 2), repeat=n):
        pat = np.array(pat)
        x = np.where(pat == 1, C, 0.0).astype(np.float64)
        F = pat == 2
        if F.any():
            lam = (np.sum(y[F] * u[F]) + C * np.sum(y[pat == 1])) / F.sum()
            x[F] = u[F] - lam * y[F]
            if np.any(x[F] < -1e-12) or np.any(x[F] > C + 1e-12):
                continue
        elif abs(np.sum(y * x)) > 1e-12:
            continue
        d = np.sum((x - u) ** 2)
        if d < best:
            best, bestx = d, x
    return bestx


@pytest.mark.parametrize("seed", range(12))
def test_projection_vs_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 8))
    C = float(rng.uniform(0.2, 3.0))
    y = rng.choice([-1, 1], size=n).astype(np.int8)
    y[0], y[1] = 1, -1
    u = rng.normal(0, 2.0, size=n)
    pi, lam = oracle.project(u, y, C)
    ref = _proj_bruteforce(u, y.astype(np.float64), C)
    np.testing.assert_allclose(pi, ref, atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_projection_kkt_large(seed):
    """KKT of the projection (eq. (3.6)): pi = Pi_K(u - lam y), y'pi = 0, and
    pi is no farther from u than random feasible points."""
    rng = np.random.default_rng(200 + seed)
    n = 5000
    y = np.where(rng.random(n) < 0.4, 1, -1).astype(np.int8)
    C = 0.7
    u = rng.normal(0.2, 1.5, size=n)
    pi, lam = oracle.project(u, y, C)
    np.testing.assert_array_equal(pi, np.clip(u - lam * y, 0.0, C))
    assert abs(np.sum(y * pi)) <= 1e-12 * np.sum(np.abs(pi))
    d0 = np.sum((pi - u) ** 2)
    for _ in range(5):
        x = _proj_bruteforce_like_feasible(rng, y, C, n)
        assert np.sum((x - u) ** 2) >= d0


def _proj_bruteforce_like_feasible(rng, y, C, n):
    # a random feasible point: equal mass on both classes
    x = rng.uniform(0, C, size=n)
    sp, sn = x[y > 0].sum(), x[y < 0].sum()
    if sp > sn:
        x[y > 0] *= sn / sp
    else:
        x[y < 0] *= sp / sn
    return x


def test_projection_breakpoint_scan():
    """grad phi is piecewise linear with breakpoints y_i(u_i - C), y_i u_i:
    evaluating it at every breakpoint and interpolating across the sign change
    gives the same lambda as Algorithm 2."""
    rng = np.random.default_rng(7)
    n, C = 9, 1.3
    y = np.array([1, -1, 1, -1, 1, 1, -1, -1, 1], np.int8)
    u = rng.normal(0.5, 1.0, size=n)
    t = np.sort(np.concatenate([y * (u - C), y * u]))
    gphi = np.array([-np.sum(y * np.clip(u - lt * y, 0, C)) for lt in t])
    k = np.nonzero(gphi >= 0)[0][0]
    lam_ref = t[k - 1] - gphi[k - 1] * (t[k] - t[k - 1]) / (gphi[k] - gphi[k - 1])
    _, lam = oracle.project(u, y, C)
    assert lam == pytest.approx(lam_ref, abs=1e-13)


# ------------------------------------------------------- HS-Jacobian / psi

def _hs_jacobian(y, J, n):
    """Theorem 3.2: P = S (I - a a'/(a'S a)) S with S = Diag(1_J), a = y."""
    S = np.zeros((n, n))
    S[J, J] = 1.0
    a = y.astype(np.float64)
    den = a @ S @ a
    if den == 0:
        return S
    return S @ (np.eye(n) - np.outer(a, a) / den) @ S


@pytest.mark.parametrize("seed", range(4))
def test_hs_jacobian_finite_difference(seed):
    rng = np.random.default_rng(300 + seed)
    n, C = 40, 1.0
    y = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    u = rng.normal(0.5, 1.0, size=n)
    pi, lam = oracle.project(u, y, C)
    J = oracle.free_set(u, y, C, lam)
    t = u - lam * y
    assert np.min(np.minimum(np.abs(t), np.abs(t - C))) > 1e-4   # away from kinks
    P = _hs_jacobian(y, J, n)
    np.testing.assert_allclose(P, P.T, atol=1e-14)
    np.testing.assert_allclose(P @ P, P, atol=1e-12)
    h = rng.normal(size=n)
    eps = 1e-7
    fd = (oracle.project(u + eps * h, y, C)[0] - oracle.project(u - eps * h, y, C)[0]) / (2 * eps)
    np.testing.assert_allclose(fd, P @ h, atol=1e-6)


def _psi_of_v(X, y, C, alpha, sigma, v):
    z = oracle.matvec(X, y, v)
    u = alpha - sigma * (z - 1.0)
    pi, _ = oracle.project(u, y, C)
    return oracle.psi(v, u, pi, alpha, sigma), pi


@pytest.mark.parametrize("seed", range(3))
def test_psi_gradient_finite_difference(seed):
    """grad_v psi = v - A'Pi(u(v)) (eq. (3.10) in q coordinates)."""
    X, y = datagen.small(60, 7, seed=seed)
    C, sigma = 0.8, 2.5
    rng = np.random.default_rng(seed)
    alpha = oracle.project(rng.uniform(0, C, 60), y, C)[0]
    v = rng.normal(0, 0.3, size=7)
    _, pi = _psi_of_v(X, y, C, alpha, sigma, v)
    g = v - (X * y[:, None]).T @ pi
    h = 1e-6
    fd = np.array([(_psi_of_v(X, y, C, alpha, sigma, v + h * e)[0]
                    - _psi_of_v(X, y, C, alpha, sigma, v - h * e)[0]) / (2 * h)
                   for e in np.eye(7)])
    np.testing.assert_allclose(fd, g, atol=2e-6)


def test_psi_is_inf_over_z():
    """psi(w) = inf_z Psi(w, z) (eq. (3.3)); the infimum is attained at
    z = (u - Pi(u))/sigma (eq. (3.4b)) and any other z gives a larger value.
    Psi is evaluated from its definition with the support function of
    K cap L computed by brute-force LP over the box plus the linear constraint
    (max over x in K cap L of <z, x> = max over lambda-shifted box vertices)."""
    rng = np.random.default_rng(11)
    n, q, C, sigma = 6, 3, 1.0, 1.7
    X, y = datagen.small(n, q, seed=3)
    alpha = oracle.project(rng.uniform(0, C, n), y, C)[0]
    A = X * y[:, None]
    w = rng.normal(size=n)
    v = A.T @ w
    u = alpha - sigma * (A @ v - 1.0)
    pi, _ = oracle.project(u, y, C)
    psi = oracle.psi(v, u, pi, alpha, sigma)

    def support(zz):
        # max <zz, x> over {0<=x<=C, y'x=0}: enumerate vertices of the polytope
        best = -np.inf
        for pat in itertools.product((0, 1, 2), repeat=n):
            pat = np.array(pat)
            if np.sum(pat == 2) > 1:
                continue
            x = np.where(pat == 1, C, 0.0)
            F = pat == 2
            if F.any():
                i = np.nonzero(F)[0][0]
                x[i] = -y[i] * np.sum(y * x)
                if x[i] < -1e-12 or x[i] > C + 1e-12:
                    continue
            elif abs(np.sum(y * x)) > 1e-12:
                continue
            best = max(best, zz @ x)
        return best

    def Psi(zz):
        Qw = A @ v
        r = Qw + zz - 1.0 - alpha / sigma
        return 0.5 * v @ v + support(zz) + 0.5 * sigma * r @ r - alpha @ alpha / (2 * sigma)

    zstar = (u - pi) / sigma
    assert Psi(zstar) == pytest.approx(psi, rel=1e-12, abs=1e-12)
    for _ in range(5):
        assert Psi(zstar + 0.05 * rng.normal(size=n)) >= psi - 1e-12


# ------------------------------------------------------------ Newton system

@pytest.mark.parametrize("n,q,seed", [(30, 5, 0), (25, 12, 1), (40, 3, 2), (18, 20, 3)])
def test_newton_forms_agree_with_nspace_system(n, q, seed):
    """Proposition 3.5: the reduced solve reproduces Q d and d'Qd of the
    n-space system (Q + sigma Q P Q) d = -grad psi, d in Ran(Q), which is
    solved here densely with a pseudo-inverse (numpy)."""
    X, y = datagen.small(n, q, seed=seed)
    rng = np.random.default_rng(seed)
    C, sigma = 1.0, 3.0
    A = X * y[:, None]
    Q = A @ A.T
    alpha = oracle.project(rng.uniform(0, C, n), y, C)[0]
    r0 = rng.normal(size=q)
    for scale in (0.2, 0.05, 0.01, 0.002):       # pick w with a proper free set
        w = A @ (scale * r0)                     # w in Ran(Q)
        v = A.T @ w
        u = alpha - sigma * (Q @ w - 1.0)
        pi, lam = oracle.project(u, y, C)
        J = oracle.free_set(u, y, C, lam)
        if 0 < J.size < n:
            break
    assert 0 < J.size < n
    g = v - A.T @ pi
    grad = Q @ w - Q @ pi
    np.testing.assert_allclose(A @ g, grad, atol=1e-10)
    P = _hs_jacobian(y, J, n)
    M = Q + sigma * Q @ P @ Q
    d = np.linalg.pinv(M, rcond=1e-13) @ (-grad)
    dv_q = oracle.newton_direction(X, y, J, sigma, g, form=1)
    dv_p = oracle.newton_direction(X, y, J, sigma, g, form=2)
    np.testing.assert_allclose(dv_q, dv_p, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(A @ dv_q, Q @ d, rtol=1e-7, atol=1e-9)        # Q d
    assert dv_q @ dv_q == pytest.approx(d @ Q @ d, rel=1e-7)                 # d'Qd


def test_newton_empty_free_set():
    """Case (b) of Proposition 3.5 with a'Sigma a = 0 (J empty): P = 0, dv = -g."""
    X, y = datagen.small(10, 4, seed=0)
    g = np.arange(4.0)
    np.testing.assert_array_equal(oracle.newton_direction(X, y, np.zeros(0, np.int64), 2.0, g), -g)


# ------------------------------------------------------ matvecs (library)

def test_matvecs_against_numpy():
    for dt in (np.float64, np.float32):
        X, y = datagen.small(300, 17, seed=5, dtype=dt)
        rng = np.random.default_rng(0)
        v, p = rng.normal(size=17), rng.normal(size=300)
        A = X.astype(np.float64) * y[:, None]
        np.testing.assert_allclose(oracle.matvec(X, y, v), A @ v, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(oracle.rmatvec(X, y, p), A.T @ p, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------- whole solves

def _qp_bruteforce(Q, y, C):
    """min 1/2 a'Qa - e'a  s.t. y'a = 0, 0 <= a <= C by enumerating every
    lower/upper/free pattern and solving the equality-constrained QP on the
    free set with a minimum-norm least-squares KKT solve."""
    n = y.size
    yf = y.astype(np.float64)
    best = np.inf
    for pat in itertools.product((0, 1, 2), repeat=n):
        pat = np.array(pat)
        U, F = pat == 1, pat == 2
        a = np.where(U, C, 0.0)
        if F.any():
            nf = F.sum()
            K = np.zeros((nf + 1, nf + 1))
            K[:nf, :nf] = Q[np.ix_(F, F)]
            K[:nf, nf] = yf[F]
            K[nf, :nf] = yf[F]
            rhs = np.concatenate([1.0 - C * Q[np.ix_(F, U)].sum(axis=1), [-C * yf[U].sum()]])
            sol, *_ = np.linalg.lstsq(K, rhs, rcond=None)
            if np.linalg.norm(K @ sol - rhs) > 1e-9 * (1 + np.linalg.norm(rhs)):
                continue
            aF = sol[:nf]
            if np.any(aF < -1e-12) or np.any(aF > C + 1e-12):
                continue
            a[F] = np.clip(aF, 0, C)
        elif abs(yf @ a) > 1e-12:
            continue
        f = 0.5 * a @ Q @ a - a.sum()
        best = min(best, f)
    return best


@pytest.mark.parametrize("n,q,seed,C", [(8, 10, 0, 1.0), (8, 3, 1, 0.5), (7, 2, 2, 5.0),
                                        (8, 5, 3, 0.3), (9, 4, 4, 2.0), (10, 6, 5, 1.0)])
def test_solve_vs_bruteforce(n, q, seed, C):
    X, y = datagen.small(n, q, seed=seed, mean_scale=1.0, flip=0.2)
    if abs(int(y.sum())) == n:
        pytest.skip("single class")
    A = X * y[:, None]
    fstar = _qp_bruteforce(A @ A.T, y, C)
    r = oracle.solve(X, y, C, tol=1e-11)
    assert r["status"] == oracle.OK
    assert r["objective"] == pytest.approx(fstar, rel=1e-9, abs=1e-10)
    assert r["kkt"] <= 1e-11


@pytest.mark.parametrize("seed", range(3))
def test_solve_invariants_and_gap(seed):
    """Every alpha^k (k >= 1) is feasible (eq. (3.5) makes it a projection),
    R_KKT reaches the tolerance, and the primal-dual gap closes."""
    X, y = datagen.small(400, 12, seed=seed, flip=0.1)
    C = 0.5
    r = oracle.solve(X, y, C, tol=1e-10, trace=True)
    assert r["status"] == oracle.OK and r["kkt"] <= 1e-10
    for t in r["trace"]:
        assert t["amin"] >= 0.0 and t["amax"] <= C
        assert abs(t["ytalpha"]) <= 1e-12 * 400 * C
    a = r["alpha"]
    assert a.min() >= 0 and a.max() <= C
    assert abs(np.sum(y * a)) <= 1e-12 * 400 * C
    # gap closes to roundoff at the tight tolerance
    assert r["gap"] <= 1e-7 * (1 + abs(r["primal"]))
    assert r["gap"] >= -1e-9 * (1 + abs(r["primal"]))
    # with free SVs the bias is unique: hinge-minimiser midpoint == KKT multiplier
    assert r["n_free"] > 0
    b, lo, hi = oracle.bias(X, y, r["w"])
    assert hi - lo <= 1e-6
    assert r["lam_kkt"] == pytest.approx(b, abs=1e-6)


def test_two_point_closed_form():
    """n = 2 (one point per class): alpha_1 = alpha_2 = t* = min(C, 2/|D|^2),
    w = t* D with D = x_1 - x_2, and b = (|x_2|^2 - |x_1|^2)/|D|^2 when t* < C."""
    x1 = np.array([1.0, 2.0, -0.5])
    x2 = np.array([-0.3, 0.4, 0.9])
    X = np.stack([x1, x2])
    y = np.array([1, -1], np.int8)
    D = x1 - x2
    for C in (10.0, 0.2):
        t = min(C, 2.0 / (D @ D))
        r = oracle.solve(X, y, C, tol=1e-12)
        assert r["status"] == oracle.OK
        np.testing.assert_allclose(r["alpha"], [t, t], rtol=1e-10)
        np.testing.assert_allclose(r["w"], t * D, rtol=1e-10)
        assert r["objective"] == pytest.approx(0.5 * t * t * (D @ D) - 2 * t, rel=1e-12)
        if t < C:
            assert r["b"] == pytest.approx((x2 @ x2 - x1 @ x1) / (D @ D), abs=1e-9)


def test_all_at_upper_bound():
    """Balanced labels and C small enough that every margin is violated at
    alpha = C e: then alpha* = C e exactly (gradient of every component is
    negative at the upper bound)."""
    X, y = datagen.small(40, 5, seed=9, mean_scale=0.2, flip=0.0)
    assert y.sum() == 0
    C = 1e-3
    w = C * (X * y[:, None]).sum(axis=0)
    assert np.max(np.abs(X @ w)) < 0.5          # |y_i <w,x_i>| < 1/2: margins all violated for |b| < 1/2
    r = oracle.solve(X, y, C, tol=1e-12)
    np.testing.assert_allclose(r["alpha"], C, rtol=0, atol=1e-15)


def test_equality_qp_when_no_bound_active():
    """With q >= n, C huge and all points support vectors, no bound is active
    at the optimum and alpha* solves the KKT system [Q y; y' 0][a; b] = [e; 0]."""
    n, q = 6, 9
    y = np.array([1, -1, 1, -1, 1, -1], np.int8)
    for seed in range(100):                      # first data set with every alpha_i > 0
        X = np.random.default_rng(seed).normal(size=(n, q))
        A = X * y[:, None]
        Q = A @ A.T
        K = np.block([[Q, y[:, None].astype(float)], [y[None, :].astype(float), np.zeros((1, 1))]])
        sol = np.linalg.solve(K, np.concatenate([np.ones(n), [0.0]]))
        a_ref = sol[:n]
        if np.all(a_ref > 0):
            break
    assert np.all(a_ref > 0)
    r = oracle.solve(X, y, 1e6, tol=1e-12)
    np.testing.assert_allclose(r["alpha"], a_ref, rtol=1e-8)
    # the equality-constraint multiplier beta = b
    assert r["lam_kkt"] == pytest.approx(sol[n], abs=1e-8)


def test_degenerate_single_class():
    X = np.ones((5, 2))
    y = np.ones(5, np.int8)
    r = oracle.solve(X, y, 1.0)
    assert r["status"] == oracle.ERR_DEGENERATE
    assert np.all(r["alpha"] == 0)


def test_kkt_zero_at_bruteforce_optimum_positive_elsewhere():
    X, y = datagen.small(8, 3, seed=1, flip=0.2)
    r = oracle.solve(X, y, 0.5, tol=1e-12)
    assert oracle.kkt(X, y, 0.5, r["alpha"]) <= 1e-12
    a = r["alpha"].copy()
    a[:2] = a[:2][::-1] + 0.01
    assert oracle.kkt(X, y, 0.5, a) > 1e-4


@pytest.mark.parametrize("ex", ["1", "2"])
def test_kkt_hand_worked_examples(ex):
    """R_KKT of eq. (4.1) on two hand-worked cases (tests/golden/kkt_worked.txt):
    the numerator's projection multiplier and the (1 + |alpha|) denominator are
    both pinned (|alpha| or 1 + |alpha|^2 in its place gives a different value)."""
    g = _read_golden("kkt_worked.txt")
    y = g["y" + ex].astype(np.int8)
    n = y.size
    X = g["X" + ex].reshape(n, -1)
    r, lam, w = oracle.kkt(X, y, g["C" + ex][0], g["alpha" + ex], with_extras=True)
    assert r == pytest.approx(g["R" + ex][0], rel=1e-14)
    assert lam == pytest.approx(g["lambda" + ex][0], abs=1e-14)
