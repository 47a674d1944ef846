"""FP64 reference of the Nystrom front-end (test infrastructure only: the
tests use it; the product path never does).

Sec. 4.3 of the paper approximates the RBF kernel matrix K (K_ij =
exp(-|x_i - x_j|^2 / (2 alpha))) from a landmark set of size r:

    K ~ K_nr K_rr^{-1} K_nr',   with K_rr replaced by K_rr + s I, s = 1e-3,

and chooses the landmarks by k-means clustering.  Readings: the landmarks are
the k-means centres (the improved Nystrom method the paper cites), found by
Lloyd's iterations from r distinct seeded rows of X; the features that make
the approximation a linear kernel are Z = K_nr L^{-T} with L L' = K_rr + s I
(Cholesky), so that Z Z' = K_nr (K_rr + s I)^{-1} K_nr' exactly.

Pinned by tests/test_nystrom_oracle.py: Z Z' against the formula with an
explicit inverse, the exact kernel recovered when every point is a landmark
and s is small, and the k-means objective and fixed point.
"""
from __future__ import annotations

import numpy as np


def rbf(A, Bm, alpha):
    """K_ij = exp(-|a_i - b_j|^2 / (2 alpha)) for the rows of A and Bm."""
    A = np.asarray(A, dtype=np.float64)
    Bm = np.asarray(Bm, dtype=np.float64)
    d2 = (A * A).sum(1)[:, None] + (Bm * Bm).sum(1)[None, :] - 2.0 * A @ Bm.T
    return np.exp(-np.maximum(d2, 0.0) / (2.0 * alpha))


def kmeans(X, r, iters=20, seed=0):
    """Lloyd's k-means from r distinct seeded rows; returns (centres, objective per step)."""
    X = np.asarray(X, dtype=np.float64)
    rng = np.random.default_rng(seed)
    cen = X[rng.choice(X.shape[0], size=r, replace=False)].copy()
    hist = []
    for _ in range(iters):
        d2 = (X * X).sum(1)[:, None] + (cen * cen).sum(1)[None, :] - 2.0 * X @ cen.T
        lab = np.argmin(d2, axis=1)
        hist.append(float(np.maximum(d2[np.arange(X.shape[0]), lab], 0.0).sum()))
        for j in range(r):
            m = lab == j
            if np.any(m):
                cen[j] = X[m].mean(axis=0)
    return cen, hist


def nystrom_features(X, centres, alpha, shift=1e-3):
    """Z = K_nr L^{-T}, L L' = K_rr + shift I (n x r)."""
    Knr = rbf(X, centres, alpha)
    Krr = rbf(centres, centres, alpha) + shift * np.eye(centres.shape[0])
    L = np.linalg.cholesky(Krr)
    return np.linalg.solve(L, Knr.T).T
