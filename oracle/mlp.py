"""FP64 reference of the learned warm start (test infrastructure only: the
tests and the CPU baseline use it; the product path never does).

The paper warm-starts SSsNAL from a random-feature solve (Sec. 4.3); the
network here predicts, per sample, whether its dual variable ends at 0, in
(0, C) or at C, from the sample and four statistics, and turns the prediction
into a starting point alpha^0 for Algorithm 1.  Everything below is the plain
definition of each step, in FP64 numpy:

  features  F_i = [x_i, y_i, |x_i|/sqrt(q), y_i (w.x_i + b)/|w|, log10 C],
            w = mu_+ - mu_- (difference of the class means), b = -w.(mu_+ + mu_-)/2
  network   Z1 = F W1 + b1, H1 = gelu(Z1), Z2 = H1 W2 + b2, H2 = gelu(Z2),
            Z3 = H2 W3 + b3 (logits of the classes 0: alpha = 0, 1: free, 2: alpha = C),
            gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2
  loss      L = (1/N) sum_i c_{l_i} (logsumexp(Z3_i) - Z3_i[l_i])  (class-weighted
            cross-entropy), and its gradient by the chain rule
  AdamW     Kingma and Ba (2015), bias-corrected moments, with the decoupled
            weight decay of Loshchilov and Hutter (2019)
  start     alpha^0_i = 0, C/2 or C for the predicted class (then projected onto
            the feasible set by the solver's warm-start path)

Pinned by tests/test_mlp_oracle.py: finite differences of L, closed forms of
gelu and of the first Adam step, and the features on a hand-checked example.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN, H, OUT = 132, 256, 3
SIZES = [(IN, H), (H,), (H, H), (H,), (H, OUT), (OUT,)]
NPARAM = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for s in SIZES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def features(X, y, C):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    mp = X[y > 0].mean(axis=0)
    mm = X[y < 0].mean(axis=0)
    w = mp - mm
    b = -w @ (mp + mm) / 2.0
    q = X.shape[1]
    nw = np.linalg.norm(w)
    marg = y * (X @ w + b) / (nw if nw > 0 else 1.0)
    return np.column_stack([X, y, np.linalg.norm(X, axis=1) / math.sqrt(q), marg,
                            np.full(X.shape[0], math.log10(C))])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_prime(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, F, keep=False):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    Z1 = F @ W1 + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2 + b2
    H2 = gelu(Z2)
    Z3 = H2 @ W3 + b3
    return (Z3, (Z1, H1, Z2, H2)) if keep else Z3


def loss(theta, F, labels, cw):
    Z3 = forward(theta, F)
    m = Z3.max(axis=1, keepdims=True)
    lse = (m + np.log(np.exp(Z3 - m).sum(axis=1, keepdims=True)))[:, 0]
    ce = lse - Z3[np.arange(F.shape[0]), labels]
    return float(np.mean(np.asarray(cw, dtype=np.float64)[labels] * ce))


def grad(theta, F, labels, cw):
    """Analytic gradient of loss() (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    Z3, (Z1, H1, Z2, H2) = forward(theta, F, keep=True)
    N = F.shape[0]
    P = np.exp(Z3 - Z3.max(axis=1, keepdims=True))
    P /= P.sum(axis=1, keepdims=True)
    D3 = P.copy()
    D3[np.arange(N), labels] -= 1.0
    D3 *= (np.asarray(cw, dtype=np.float64)[labels] / N)[:, None]
    gW3, gb3 = H2.T @ D3, D3.sum(axis=0)
    D2 = (D3 @ W3.T) * gelu_prime(Z2)
    gW2, gb2 = H1.T @ D2, D2.sum(axis=0)
    D1 = (D2 @ W2.T) * gelu_prime(Z1)
    gW1, gb1 = F.T @ D1, D1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (t = 1, 2, ...): Adam's bias-corrected step plus the
    decoupled weight decay lr * wd * theta of Loshchilov and Hutter (2019);
    returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta), m, v


def classes_of(alpha, C):
    """Labels harvested from a solution: 0 (alpha = 0), 2 (alpha = C), 1 (free)."""
    alpha = np.asarray(alpha)
    return np.where(alpha <= 0.0, 0, np.where(alpha >= C, 2, 1)).astype(np.int32)


def start_point(logits, C):
    """alpha^0 from the predicted classes: 0, C/2, C."""
    cls = np.argmax(logits, axis=1)
    return np.choose(cls, [0.0, 0.5 * C, C])
