"""Pins of the random Fourier features reference (oracle/rff.py) against
what the mathematics fixes, independently of its own formula."""
import numpy as np

import datagen
from oracle import rff


def _data(n=40, q=7, N=33, alpha=2.5, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, q))
    Om = datagen.rff_omega(seed, q, N, alpha).astype(np.float64)
    return X, Om


def test_rows_have_unit_norm():
    # cos^2 + sin^2 = 1 per frequency, N frequencies, 1/sqrt(N) scaling: |z(x)| = 1 = k(x, x)
    X, Om = _data()
    Z = rff.rff_features(X, Om)
    np.testing.assert_allclose(np.linalg.norm(Z, axis=1), 1.0, rtol=0, atol=1e-14)


def test_inner_products_are_the_sample_average_of_cos_of_differences():
    # z(x)'z(y) = (1/N) sum_j cos(omega_j'(x - y)) (cos a cos b + sin a sin b = cos(a - b)),
    # evaluated here from the difference vectors, not from the features
    X, Om = _data(n=12)
    Z = rff.rff_features(X, Om)
    N = Om.shape[1]
    for i in range(12):
        for j in range(12):
            direct = np.cos((X[i] - X[j]) @ Om).sum() / N
            assert abs(Z[i] @ Z[j] - direct) <= 1e-13


def test_monte_carlo_estimate_of_the_rbf_kernel():
    # E[cos(omega'd)] = exp(-|d|^2 / (2 alpha)) for omega ~ N(0, I/alpha): at N = 2^16 the
    # sample average is within 5 standard errors (std of cos <= 1) of the kernel
    alpha, q, N = 1.7, 5, 1 << 16
    rng = np.random.default_rng(3)
    X = rng.normal(size=(6, q)) * 0.8
    Om = datagen.rff_omega(11, q, N, alpha).astype(np.float64)
    Z = rff.rff_features(X, Om)
    for i in range(6):
        for j in range(6):
            assert abs(Z[i] @ Z[j] - rff.rbf_kernel(X[i], X[j], alpha)) <= 5.0 / np.sqrt(N)


def test_frequencies_have_the_stated_distribution():
    # omega ~ N(0, I/alpha): sample variance alpha^{-1} within 3% at 2^16 draws
    Om = datagen.rff_omega(5, 4, 1 << 14, 0.5).astype(np.float64)
    assert abs(Om.var() * 0.5 - 1.0) <= 0.03
    assert abs(Om.mean()) <= 0.03
