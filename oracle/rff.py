"""FP64 reference of the random Fourier features front-end (test
infrastructure only: the tests use it; the product path never does).

Sec. 4.3 of the paper approximates the RBF kernel k(x, y) = exp(-|x - y|^2 /
(2 alpha)) by Bochner's theorem: with omega_1 .. omega_N drawn independently
from the Gaussian density proportional to exp(-alpha |omega|^2 / 2) (that is,
N(0, I / alpha)), the map

    z(x) = [cos(omega_1' x), sin(omega_1' x), ..., cos(omega_N' x), sin(omega_N' x)] / sqrt(N)

gives z(x)' z(y) = (1/N) sum_j cos(omega_j' (x - y)), the sample average whose
expectation is k(x, y).  The rows z(x_i) form the n x 2N matrix Z_omega that
replaces X in the linear C-SVC dual.  Reading: the paper writes K ~ Z Z'
without the 1/N of the sample average it states just before; the map here
carries 1/sqrt(N) so that Z Z' is that average (the scale only reparametrises
C otherwise).

Pinned by tests/test_rff_oracle.py: unit rows (cos^2 + sin^2 = 1), the
inner-product identity against a direct sum over omega' (x - y), and the
Monte-Carlo agreement with exp(-|x - y|^2 / (2 alpha)) at large N.
"""
from __future__ import annotations

import numpy as np


def rff_features(X, Omega):
    """Z (n x 2N, FP64) from X (n x q) and Omega (q x N, columns omega_j)."""
    X = np.asarray(X, dtype=np.float64)
    Om = np.asarray(Omega, dtype=np.float64)
    N = Om.shape[1]
    T = X @ Om                      # T_ij = omega_j' x_i
    Z = np.empty((X.shape[0], 2 * N), dtype=np.float64)
    Z[:, 0::2] = np.cos(T)
    Z[:, 1::2] = np.sin(T)
    return Z / np.sqrt(N)


def rbf_kernel(x, y, alpha):
    """k(x, y) = exp(-|x - y|^2 / (2 alpha)) (the paper's RBF kernel, read with
    the 2 alpha in the denominator)."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    return float(np.exp(-(d @ d) / (2.0 * alpha)))
