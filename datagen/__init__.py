"""Seeded synthetic inputs for the linear C-SVC dual (arXiv 1910.01312).

This module only draws data; it holds none of the method's arithmetic.  Both
the FP64 oracle (tests, CPU baseline) and the CUDA path read the arrays it
returns, so the two sides always see the same bytes.

The paper evaluates on LIBSVM datasets (Sec. 4, Table 1), which are not
available here; the workloads below stand in for them with the shapes, value
distributions and label structure of a two-class problem with label noise.
Every generator is keyed by (workload id, seed) through numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

_IDS = {"small": 0, "gauss2000": 1, "gauss1m": 2, "csr": 3, "mnist_like": 4, "warm": 5, "ovr": 6, "rff": 7}


def _rng(kind: str, seed: int) -> np.random.Generator:
    return np.random.default_rng([_IDS[kind], int(seed)])


def balanced_labels(rng: np.random.Generator, n: int) -> np.ndarray:
    """n/2 (+1) and n - n/2 (-1) labels in random order, int8."""
    y = np.empty(n, np.int8)
    y[: (n + 1) // 2] = 1
    y[(n + 1) // 2:] = -1
    rng.shuffle(y)
    return y


def flip_labels(rng: np.random.Generator, y: np.ndarray, frac: float) -> np.ndarray:
    """Flip exactly round(frac*n) labels chosen uniformly without replacement."""
    y = y.copy()
    k = int(round(frac * y.size))
    if k:
        idx = rng.choice(y.size, size=k, replace=False)
        y[idx] = -y[idx]
    return y


def gaussian_two_class(n: int, q: int, mean_scale: float, var=None, flip: float = 0.0,
                       seed: int = 0, dtype=np.float64, kind: str = "small"):
    """Rows x_i = y_i * mean_scale/sqrt(q) * 1 + sqrt(var) * eps_i, eps ~ N(0, I_q),
    drawn with the true label, then a fraction `flip` of the labels flipped.

    Returns (X [n x q, row-major, dtype], y [n] int8 in {-1,+1})."""
    rng = _rng(kind, seed)
    y_true = balanced_labels(rng, n)
    mu = mean_scale / np.sqrt(q)
    sd = np.ones(q) if var is None else np.sqrt(np.asarray(var, dtype=np.float64))
    X = np.empty((n, q), dtype=dtype)
    step = 1 << 16
    for s in range(0, n, step):
        e = rng.standard_normal((min(step, n - s), q))
        X[s:s + e.shape[0]] = (y_true[s:s + e.shape[0], None] * mu + e * sd).astype(dtype)
    y = flip_labels(rng, y_true, flip)
    return X, y


def small(n: int, q: int, seed: int = 0, dtype=np.float64, mean_scale: float = 1.0,
          flip: float = 0.1):
    """Small random two-class problem for unit tests."""
    return gaussian_two_class(n, q, mean_scale, None, flip, seed, dtype, "small")


def gauss2000(seed: int = 0):
    """n=2000 x q=50 dense FP64, N(+-0.5/sqrt(q) 1, I), balanced, 5% flipped, C=1."""
    X, y = gaussian_two_class(2000, 50, 0.5, None, 0.05, seed, np.float64, "gauss2000")
    return X, y, 1.0


def gauss1m(seed: int = 0, n: int = 1_000_000, q: int = 128):
    """n=1e6 x q=128 dense FP32, means +-0.3/sqrt(q) 1, covariance
    diag(linspace(0.1, 2, q)), 10% labels flipped, C=0.1.  `n` may be lowered
    for bounded samples of the same distribution."""
    X, y = gaussian_two_class(n, q, 0.3, np.linspace(0.1, 2.0, q), 0.10, seed, np.float32,
                              "gauss1m")
    return X, y, 0.1


def warm_instance(seed: int, n: int = 100_000, q: int = 128, m_range=(0.1, 0.5), noise_max: float = 0.15):
    """One instance of the learned-warm-start workload: the gauss1m generator
    with per-instance class-mean scale m ~ U[m_range], label noise ~ U[0,
    noise_max] and C = 10^U[-2, 1] (the defaults: overlapping, noisy classes,
    most samples support vectors; m_range = (1, 2), noise_max = 0.01: nearly
    separable classes, few support vectors).  Returns (X [n x q] FP32, y
    int8, C)."""
    rng = _rng("warm", seed)
    m = rng.uniform(*m_range)
    noise = rng.uniform(0.0, noise_max)
    C = float(10.0 ** rng.uniform(-2.0, 1.0))
    X, y = gaussian_two_class(n, q, m, np.linspace(0.1, 2.0, q), noise, 10_000 + int(seed), np.float32, "warm")
    return X, y, C


MLP_IN, MLP_H = 132, 256          # the warm-start network: 132 -> 256 -> 256 -> 3


def mlp_init(seed: int = 0) -> np.ndarray:
    """Initial parameters of the warm-start MLP as one flat FP32 vector in the
    layout [W1 (132x256, row-major in x out), b1, W2 (256x256), b2, W3 (256x3),
    b3]: weights ~ N(0, 2/fan_in) (He), biases 0."""
    rng = np.random.default_rng([_IDS["warm"], 1_000_000 + int(seed)])
    parts = []
    for fi, fo in ((MLP_IN, MLP_H), (MLP_H, MLP_H), (MLP_H, 3)):
        parts.append((rng.standard_normal((fi, fo)) * np.sqrt(2.0 / fi)).ravel())
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def sparse_text(seed: int = 0, n: int = 700_000, q: int = 47_000, nnz_row: int = 75, zipf: float = 1.1,
                noise: float = 0.1, density_w: float = 0.1, dtype=np.float32):
    """Text-like sparse two-class problem in CSR form: each row holds nnz_row
    distinct columns drawn without replacement from a Zipf(zipf) law over the
    q columns (successive draws, repeats discarded; at most 3 nnz_row draws,
    so a row can fall short when q is small), column indices strictly
    increasing, values lognormal(0, 1), each row scaled to unit L2 norm;
    labels sign(X w* + noise eps) with w* nonzero (N(0, 1)) on a random
    density_w fraction of the columns, eps ~ N(0, 1); C = 1.

    Returns (indptr int64 [n+1], indices int32 [nnz], values dtype [nnz],
    y int8 [n], C)."""
    rng = _rng("csr", seed)
    pr = 1.0 / np.arange(1, q + 1, dtype=np.float64) ** zipf
    cdf = np.cumsum(pr)
    cdf /= cdf[-1]
    perm = rng.permutation(q)            # which column gets which frequency rank
    indptr = np.zeros(n + 1, np.int64)
    idx_parts, val_parts = [], []
    step = 1 << 15
    for s in range(0, n, step):
        m = min(step, n - s)
        K = 3 * nnz_row
        D = perm[np.minimum(np.searchsorted(cdf, rng.random((m, K))), q - 1)]
        order = np.argsort(D, axis=1, kind="stable")
        Ds = np.take_along_axis(D, order, axis=1)
        fs = np.ones_like(Ds, dtype=bool)
        fs[:, 1:] = Ds[:, 1:] != Ds[:, :-1]
        first = np.zeros_like(fs)
        np.put_along_axis(first, order, fs, axis=1)          # first draw of each column
        keep = first & (np.cumsum(first, axis=1) <= nnz_row)   # the first nnz_row distinct
        cols = np.where(keep, D, q)
        cols.sort(axis=1)
        cols = cols[:, :nnz_row]
        valid = cols < q
        cnt = valid.sum(axis=1)
        c = cols[valid].astype(np.int32)
        v = rng.lognormal(0.0, 1.0, c.size)
        starts = np.concatenate([[0], np.cumsum(cnt)[:-1]])
        norms = np.sqrt(np.add.reduceat(v * v, starts))
        v /= np.repeat(norms, cnt)
        indptr[s + 1:s + m + 1] = indptr[s] + np.cumsum(cnt)
        idx_parts.append(c)
        val_parts.append(v.astype(dtype))
    indices = np.concatenate(idx_parts)
    values = np.concatenate(val_parts)
    w = np.where(rng.random(q) < density_w, rng.standard_normal(q), 0.0)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    margin = np.bincount(rows, weights=values.astype(np.float64) * w[indices], minlength=n)
    y = np.where(margin + noise * rng.standard_normal(n) >= 0.0, 1, -1).astype(np.int8)
    return indptr, indices, values, y, 1.0


def ovr_path(seed: int = 0, n: int = 200_000, q: int = 784, n_classes: int = 10, n_C: int = 16,
             density: float = 0.2, C_lo: float = -3.0, C_hi: float = 2.0, dtype=np.float32):
    """Many SVMs over one data matrix: one-vs-rest problems of a multi-class
    labelling, each on a path of C values.

    X: n x q, each entry 0 with probability 1 - density, else U[0, 1] (an
    image-like sparse nonnegative matrix, stored dense).  Class proportions
    p ~ Dirichlet(0.5 * 1), labels c_i ~ Categorical(p), redrawn until every
    class occurs.  Problem (c, j) has y_i = +1 iff c_i = c and C = 10^(C_lo +
    (C_hi - C_lo) j / (n_C - 1)); the labels do not depend on X.

    Returns (X, Y [n_classes * n_C x n] int8, C [n_classes * n_C] float64),
    problems ordered class-major."""
    rng = _rng("ovr", seed)
    X = np.zeros((n, q), dtype=dtype)
    step = max(1, (1 << 22) // q)
    for s in range(0, n, step):
        m = min(step, n - s)
        vals = rng.random((m, q))
        keep = rng.random((m, q)) < density
        X[s:s + m] = np.where(keep, vals, 0.0).astype(dtype)
    while True:
        props = rng.dirichlet(0.5 * np.ones(n_classes))
        c = rng.choice(n_classes, size=n, p=props)
        if np.unique(c).size == n_classes:
            break
    Cs = 10.0 ** (C_lo + (C_hi - C_lo) * np.arange(n_C) / max(1, n_C - 1))
    Y = np.empty((n_classes * n_C, n), np.int8)
    Cv = np.empty(n_classes * n_C, np.float64)
    for k in range(n_classes):
        yk = np.where(c == k, 1, -1).astype(np.int8)
        for j in range(n_C):
            Y[k * n_C + j] = yk
            Cv[k * n_C + j] = Cs[j]
    return X, Y, Cv


def rff_omega(seed: int, q: int, N: int, alpha: float, dtype=np.float32):
    """The N frequencies of random Fourier features for the RBF kernel
    exp(-|x - y|^2 / (2 alpha)): columns omega_j ~ N(0, I_q / alpha), returned
    as a q x N matrix (row-major) in dtype; both sides read these values."""
    rng = _rng("rff", seed)
    return (rng.standard_normal((q, N)) / np.sqrt(alpha)).astype(dtype)
