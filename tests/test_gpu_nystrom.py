"""GPU parity of the Nystrom front-end (Sec. 4.3; include/svm_nystrom.h)
against the FP64 reference oracle/nystrom.py (pinned in
test_nystrom_oracle.py by the explicit-inverse formula, exact recovery with
every point a landmark, and the k-means fixed point).

k-means decides integers (the nearest centre) from floating point: both
sides decide in FP64; rows whose two nearest centres are within roundoff of
each other may go either way and are excluded from the exact comparison, and
the workloads below are separated blobs, so whole runs match.  Features are
compared elementwise: FP64 output within the rounding of an r-term
triangular product scaled by the factor's condition number; FP32 output
within one FP32 rounding more.  The solve on the features is compared with
the oracle's solve on the reference features through the envelope bound
|w| sum_i alpha_i |dz_i| (dz the measured feature difference).
"""
import numpy as np
import pytest

import oracle
from oracle import nystrom as ny

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


def _blobs(seed, n, q, k, spread=0.4):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-4.0, 4.0, size=(k, q))
    lab = rng.integers(0, k, size=n)
    X = (means[lab] + spread * rng.normal(size=(n, q))).astype(np.float32)
    return X, lab


def _d2(X, Cn):
    Xd = X.astype(np.float64)
    return ((Xd[:, None, :] - Cn[None, :, :]) ** 2).sum(-1)


@pytest.mark.parametrize("n,q,r", [(3000, 16, 8), (777, 3, 50), (5000, 130, 40), (64, 1024, 5)])
def test_kmeans_step_matches_the_definition(n, q, r):
    """One Lloyd step: each row goes to its nearest centre (FP64 distances,
    ties to the lowest index), each centre becomes the mean of its rows."""
    X, _ = _blobs(n + q, n, q, max(2, r // 2))
    rng = np.random.default_rng(1)
    C0 = X[rng.choice(n, size=r, replace=False)].astype(np.float64)
    Cd = dev(C0)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    obj = P.nystrom_kmeans(dev(X), Cd, 1, labels=lab)
    d2 = _d2(X, C0)
    lr = np.argmin(d2, axis=1)
    lg = host(lab)
    srt = np.sort(d2, axis=1)
    tie = (srt[:, 1] - srt[:, 0]) <= 1e-12 * (1.0 + srt[:, 1]) if r > 1 else np.zeros(n, bool)
    assert np.all((lg == lr) | tie)
    assert obj[0] == pytest.approx(d2[np.arange(n), lg].sum(), rel=1e-12)
    C1 = host(Cd)
    Xd = X.astype(np.float64)
    for j in range(r):
        m = lg == j
        want = Xd[m].mean(axis=0) if m.any() else C0[j]
        np.testing.assert_allclose(C1[j], want, rtol=1e-13, atol=1e-13 * (1 + np.abs(want).max()))


def test_kmeans_iterations_match_reference():
    X, _ = _blobs(7, 4000, 10, 6)
    r, iters, seed = 6, 12, 5
    cen_r, hist_r = ny.kmeans(X, r, iters=iters, seed=seed)
    rng = np.random.default_rng(seed)                  # the reference's initial centres
    C0 = X[rng.choice(X.shape[0], size=r, replace=False)].astype(np.float64)
    Cd = dev(C0)
    hist = P.nystrom_kmeans(dev(X), Cd, iters)
    np.testing.assert_allclose(hist, hist_r, rtol=1e-10)
    np.testing.assert_allclose(host(Cd), cen_r, rtol=0, atol=1e-12 * (1 + np.abs(cen_r).max()))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:]))


def _feature_bound(Z_ref, Krr):
    # Z = K_nr L^{-T} through the computed inverse factor: r-term FP64 sums whose
    # error is at most r u cond(L)^2 = r u cond(K_rr + s I) relative to |Z| (with margin)
    r = Krr.shape[0]
    return 8.0 * r * 2.0 ** -53 * np.linalg.cond(Krr) * (1.0 + np.abs(Z_ref).max())


@pytest.mark.parametrize("n,q,r,alpha", [(5000, 20, 64, 2.0), (1001, 7, 33, 0.5), (3000, 128, 256, 40.0),
                                         (100, 5, 1, 1.0)])
def test_features_match_reference(n, q, r, alpha):
    rng = np.random.default_rng(n + r)
    X = rng.normal(size=(n, q)).astype(np.float32)
    Cn = X[rng.choice(n, size=r, replace=False)].astype(np.float64) + 0.01 * rng.normal(size=(r, q))
    Zr = ny.nystrom_features(X, Cn, alpha, 1e-3)
    Krr = ny.rbf(Cn, Cn, alpha) + 1e-3 * np.eye(r)
    bound = _feature_bound(Zr, Krr)
    Z64 = torch.empty((n, r), dtype=torch.float64, device="cuda")
    P.nystrom_features(dev(X), dev(Cn), alpha, Z64)
    np.testing.assert_allclose(host(Z64), Zr, rtol=0, atol=bound)
    Z32 = torch.empty((n, r), dtype=torch.float32, device="cuda")
    P.nystrom_features(dev(X), dev(Cn), alpha, Z32)
    np.testing.assert_allclose(host(Z32).astype(np.float64), Zr, rtol=2.0 ** -24, atol=bound)
    # the approximation itself: Z Z' = K_nr (K_rr + s I)^{-1} K_nr' on a few rows
    Knr = ny.rbf(X[:40], Cn, alpha)
    ref = Knr @ np.linalg.solve(Krr, Knr.T)
    Zg = host(Z64)[:40]
    np.testing.assert_allclose(Zg @ Zg.T, ref, rtol=0, atol=1e-9 * np.linalg.cond(Krr))


def test_solve_on_gpu_features_matches_oracle_on_reference_features():
    """The RBF C-SVC through Nystrom features, the way Sec. 4.3 uses them:
    k-means landmarks, K_rr + 1e-3 I, then the linear solver on Z."""
    import datagen
    X, y = datagen.small(4000, 10, seed=9, dtype=np.float32, mean_scale=1.5)
    r, alpha, C = 64, 4.0, 1.0
    rng = np.random.default_rng(3)
    Cd = dev(X[rng.choice(X.shape[0], size=r, replace=False)].astype(np.float64))
    Xd = dev(X)
    P.nystrom_kmeans(Xd, Cd, 10)
    Z = torch.empty((X.shape[0], r), dtype=torch.float32, device="cuda")
    P.nystrom_features(Xd, Cd, alpha, Z)
    n = X.shape[0]
    s = P.Solver(Z, dev(y.astype(np.int8)), C_=C, tol=1e-6, precision=P.PREC_MIXED)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(r, dtype=torch.float64, device="cuda")
    res = s.solve(a, w)
    s.close()
    assert res["status"] == P.OK and res["kkt"] <= 1e-6 and res["form"] == P.FORM_MIXED
    Zr = ny.nystrom_features(X, host(Cd), alpha, 1e-3)
    ref = oracle.solve(Zr, y, C, tol=1e-10)
    alpha_g = host(a)
    dz = np.linalg.norm(host(Z).astype(np.float64) - Zr, axis=1)
    env = np.linalg.norm(ref["w"]) * float(np.maximum(alpha_g, ref["alpha"]) @ dz)
    assert abs(res["objective"] - ref["objective"]) <= 2e-6 * abs(ref["objective"]) + 2.0 * env
    assert oracle.kkt(Zr, y, C, alpha_g) <= 1e-5


def test_invalid_arguments():
    X = torch.ones((8, 3), dtype=torch.float32, device="cuda")
    Cn = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    Z = torch.empty((8, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(P.SVMError) as e:
        P.nystrom_features(X, Cn, -1.0, Z)
    assert e.value.status == P.ERR_INVALID_ARG
    with pytest.raises(P.SVMError) as e:                # two identical landmarks and no shift: K_rr is singular
        P.nystrom_features(X, Cn, 1.0, Z, shift=0.0)
    assert e.value.status == P.ERR_NUMERIC
    big = torch.zeros((1025, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.SVMError) as e:
        P.nystrom_kmeans(X, big, 1)
    assert e.value.status == P.ERR_UNSUPPORTED
