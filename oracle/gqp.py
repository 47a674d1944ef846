"""FP64 reference of SSsNAL for the paper's unified QP (test infrastructure
only: the tests use it; the product path never does).

The problem (Sec. 1, eq. (1.5)):

    min_x  1/2 x'Qx + c'x   s.t.  a'x = d,  l <= x <= u,     Q = B B'

with B an n x q matrix (so that the method can run in the coordinates
v = B'w of q-space, as the C-SVC solver does), any c, any a (signs and
magnitudes free, components may be 0), l < u and any d for which the set is
non-empty.  The C-SVC dual is the case B = Diag(y) X, c = -e, a = y, d = 0,
l = 0, u = C e; the SVR dual (eq. (1.4)) with the linear kernel K = X X' is
B = [X; -X], c = [eps + y; eps - y], a = [e; -e], d = 0, l = 0, u = C e
(2n variables).

The method, step by step in the paper's order:

  Alg. 1   x^{k+1} = Pi(u(w^{k+1})) (eq. (3.5)), u(w) = x^k - sigma (Q w + c),
           sigma schedule and stopping tests read as in the C-SVC oracle;
  psi      psi(w) = 1/2 <w, Qw> + (|u|^2 - |u - Pi(u)|^2) / (2 sigma) - |x^k|^2 / (2 sigma)
           (eq. (3.3)), in q-space 1/2 |v|^2 + pi'(2u - pi) / (2 sigma) - |x^k|^2 / (2 sigma);
  grad     grad psi = Q (w - Pi(u)), in q-space g = v - B' pi (eq. (3.10));
  Alg. 2   Pi onto {a'x = d, l <= x <= u}: x_i = clip(u_i - lambda a_i, l_i, u_i), lambda the
           root of the monotone piecewise-linear a'x(lambda) - d, found by sorting the
           breakpoints, bisection between them and interpolation on the last piece;
  Thm 3.2  HS-Jacobian on the free set J: P = Diag(theta) - (theta a)(theta a)' / (a_J'a_J);
  Alg. 3   Newton direction from (I + sigma B'PB) dv = -g, solved exactly (q-form,
           the matrix is SPD), Armijo line search on psi.

KKT residual (eq. (4.1)): |x - Pi(x - Qx - c)| / (1 + |x|).

Pinned by tests/test_gqp_oracle.py: the projection against an enumeration of
its optimality patterns, the C-SVC case against the C oracle, tiny problems
against an enumeration of the QP's active sets, and the SVR case by its zero
primal-dual gap with the primal objective evaluated directly.
"""
from __future__ import annotations

import numpy as np


def project(uu, a, d, lo, hi):
    """Pi_{K cap L}(uu) by Algorithm 2 (general a): returns (x, lam)."""
    uu = np.asarray(uu, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    nz = a != 0.0

    def xs(lam):
        return np.clip(uu - lam * a, lo, hi)

    def f(lam):   # a'x(lam) - d, nonincreasing in lam
        return float(a @ xs(lam)) - d

    if not np.any(nz):
        return np.clip(uu, lo, hi), 0.0
    # breakpoints: u_i - lam a_i = l_i or = u_i
    t = np.concatenate([(uu[nz] - lo[nz]) / a[nz], (uu[nz] - hi[nz]) / a[nz]])
    t = np.sort(t)
    fl, fu = f(t[0]), f(t[-1])
    if fl < 0.0 or fu > 0.0:
        raise ValueError("the set {a'x = d, l <= x <= u} is empty")
    il, iu = 0, t.size - 1
    while iu - il > 1:
        im = (il + iu) // 2
        fm = f(t[im])
        if fm > 0.0:
            il, fl = im, fm
        elif fm < 0.0:
            iu, fu = im, fm
        else:
            return xs(t[im]), float(t[im])
    tl, tu = t[il], t[iu]
    if fl == fu:
        lam = tl
    else:
        lam = tl - fl * (tu - tl) / (fu - fl)   # f is linear on [tl, tu]
    return xs(lam), float(lam)


def free_set(uu, a, lo, hi, lam):
    """J = {i : l_i < u_i - lam a_i < u_i} (ties go to the bound)."""
    r = uu - lam * np.asarray(a, dtype=np.float64)
    return np.nonzero((r > lo) & (r < hi))[0]


def kkt(B, c, a, d, lo, hi, x):
    """Relative KKT residual of eq. (4.1)."""
    Qx = B @ (B.T @ x)
    px, _ = project(x - Qx - c, a, d, lo, hi)
    return float(np.linalg.norm(x - px) / (1.0 + np.linalg.norm(x)))


def objective(B, c, x):
    w = B.T @ x
    return float(0.5 * w @ w + c @ x)


def newton_direction(B, a, J, sigma, g):
    """(I + sigma B'PB) dv = -g with P the HS-Jacobian on J (Thm. 3.2)."""
    q = B.shape[1]
    if J.size == 0:
        return -g
    BJ = B[J]
    aJ = a[J]
    M = np.eye(q) + sigma * (BJ.T @ BJ)
    ata = float(aJ @ aJ)
    if ata > 0.0:
        h = BJ.T @ aJ
        M -= sigma * np.outer(h, h) / ata
    return np.linalg.solve(M, -g)


def solve(B, c, a, d, lo, hi, tol=1e-8, sigma0=1.0, growth=5.0, sigma_max=1e6, max_outer=200,
          max_inner=50, max_ls=40, mu=1e-4, delta=0.5):
    """SSsNAL (Algorithm 1 with Algorithm 3 inside) from x^0 = 0, w^0 = 0."""
    B = np.asarray(B, dtype=np.float64)
    c, a = np.asarray(c, dtype=np.float64), np.asarray(a, dtype=np.float64)
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    n, q = B.shape
    x = np.zeros(n)
    v = np.zeros(q)
    sigma = sigma0
    R = kkt(B, c, a, d, lo, hi, x)
    Rprev = R
    k = 0
    inner_total = 0
    status = "not_converged"
    if R <= tol:
        status = "ok"
    while status != "ok" and k < max_outer:
        eps_k = 0.1 * 0.5 ** k

        def at(vv):
            uu = x - sigma * (B @ vv + c)
            pi, lam = project(uu, a, d, lo, hi)
            psi = 0.5 * vv @ vv + pi @ (2.0 * uu - pi) / (2.0 * sigma) - x @ x / (2.0 * sigma)
            return uu, pi, lam, psi

        uu, pi, lam, psi = at(v)
        for j in range(max_inner + 1):
            g = v - B.T @ pi
            scale = np.linalg.norm(np.abs(B).T @ np.abs(pi)) + np.linalg.norm(v)
            tol_in = max(min(eps_k, eps_k * np.linalg.norm(pi - x)) / np.sqrt(sigma), 1e-15 * scale)
            if np.linalg.norm(g) <= tol_in or j == max_inner:
                break
            J = free_set(uu, a, lo, hi, lam)
            dv = newton_direction(B, a, J, sigma, g)
            slope = float(g @ dv)
            t = 1.0
            accepted = False
            for _ in range(max_ls):
                ut, pit, lamt, psit = at(v + t * dv)
                if psit <= psi + mu * t * slope:
                    accepted = True
                    break
                t *= delta
            if not accepted:
                break
            v = v + t * dv
            uu, pi, lam, psi = ut, pit, lamt, psit
            inner_total += 1
        x = pi
        R = kkt(B, c, a, d, lo, hi, x)
        k += 1
        if R <= tol:
            status = "ok"
            break
        if R > 0.5 * Rprev:
            sigma = min(sigma_max, growth * sigma)
        Rprev = R
    return {"x": x, "objective": objective(B, c, x), "kkt": R, "outer": k, "inner_total": inner_total,
            "status": status, "sigma": sigma}


def svr_problem(X, y, eps, C):
    """The SVR dual (eq. (1.4)) with the linear kernel K = X X', as a unified QP in
    the variables [x; z] (2n): B = [X; -X], c = [eps + y; eps - y], a = [e; -e],
    d = 0, l = 0, u = C."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    B = np.vstack([X, -X])
    c = np.concatenate([eps + y, eps - y])
    a = np.concatenate([np.ones(n), -np.ones(n)])
    return B, c, a, 0.0, np.zeros(2 * n), np.full(2 * n, float(C))


def svr_primal(X, y, eps, C, w):
    """min over b of the SVR primal objective 1/2 |w|^2 + C sum_i max(0, |y_i - w'x_i - b| - eps)
    (eq. (1.3) with the slacks eliminated); exact, by trying every kink of the
    convex piecewise-linear function of b."""
    r = np.asarray(y, dtype=np.float64) - np.asarray(X, dtype=np.float64) @ w
    kinks = np.concatenate([r - eps, r + eps])
    vals = [np.maximum(0.0, np.abs(r - b) - eps).sum() for b in kinks]
    i = int(np.argmin(vals))
    return float(0.5 * w @ w + C * vals[i]), float(kinks[i])
