"""Pins of the Nystrom reference (oracle/nystrom.py) against results fixed
independently of its own formula."""
import numpy as np

from oracle import nystrom as ny


def test_features_reproduce_the_nystrom_approximation():
    # Z Z' = K_nr (K_rr + s I)^{-1} K_nr', here with an explicit inverse instead of
    # the Cholesky solve
    rng = np.random.default_rng(0)
    X = rng.normal(size=(50, 4))
    C = rng.normal(size=(9, 4))
    alpha, s = 1.3, 1e-3
    Z = ny.nystrom_features(X, C, alpha, s)
    Knr = np.exp(-((X[:, None, :] - C[None, :, :]) ** 2).sum(-1) / (2 * alpha))
    Krr = np.exp(-((C[:, None, :] - C[None, :, :]) ** 2).sum(-1) / (2 * alpha))
    ref = Knr @ np.linalg.inv(Krr + s * np.eye(9)) @ Knr.T
    np.testing.assert_allclose(Z @ Z.T, ref, rtol=0, atol=1e-11)


def test_every_point_a_landmark_recovers_the_kernel():
    # r = n landmarks and a tiny shift: K_nn (K_nn + s I)^{-1} K_nn = K - s I + O(s^2 / lambda_min)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(12, 3)) * 3.0          # well separated: K close to I, well conditioned
    alpha, s = 1.0, 1e-9
    Z = ny.nystrom_features(X, X, alpha, s)
    K = np.exp(-((X[:, None, :] - X[None, :, :]) ** 2).sum(-1) / (2 * alpha))
    np.testing.assert_allclose(Z @ Z.T, K, rtol=0, atol=1e-7)
    np.testing.assert_allclose(np.diag(Z @ Z.T), 1.0, rtol=0, atol=1e-7)   # k(x, x) = 1


def test_kmeans_objective_falls_and_centres_are_cluster_means():
    rng = np.random.default_rng(2)
    blobs = np.concatenate([rng.normal(loc=m, scale=0.3, size=(40, 2)) for m in ((0, 0), (4, 0), (0, 4))])
    cen, hist = ny.kmeans(blobs, 3, iters=15, seed=5)
    assert all(b <= a + 1e-9 for a, b in zip(hist, hist[1:]))
    lab = np.argmin(((blobs[:, None, :] - cen[None]) ** 2).sum(-1), axis=1)
    for j in range(3):
        np.testing.assert_allclose(cen[j], blobs[lab == j].mean(axis=0), rtol=0, atol=1e-12)
    # the three blobs are found
    assert sorted(np.bincount(lab, minlength=3).tolist()) == [40, 40, 40]
