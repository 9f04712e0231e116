"""Learned start block: vertex features, the MLP, its loss and gradients, FP64 numpy.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Not in the paper; an extension of its random start block.  A small MLP maps per-vertex
features computed with SpMM (Section 3.3) to an n x b block that starts the Block Krylov-Schur
iteration instead of a random block (Table 1, MvRandom).

Features (8 per vertex; rms(x) = sqrt(mean(x^2)), 1 when that is 0):
  d   = A 1                    (degrees)
  f0  = log(1 + d)
  f1  = d / rms(d)
  f2  = A d / rms(A d)
  f3  = A^2 d / rms(A^2 d)
  R   = N(0,1) n x 4 probe block (counter RNG, stream 6)
  q_p = mean over the 4 probe columns of (A^p R)^2, an estimate of diag(A^(2p)), p = 2, 3, 4
  f4  = q2 / rms(q2),  f5 = q3 / rms(q3),  f6 = q4 / rms(q4),  f7 = log(1 + q2 / mean(q2))

Network (hidden width H): h1 = relu(F W1 + b1), h2 = relu(h1 W2 + b2), Z = h2 W3 + b3.
Parameters are packed as [W1 (8 x H), b1 (H), W2 (H x H), b2 (H), W3 (H x b), b3 (b)], row-major.

Loss against reference Ritz vectors U (n x b, unit columns), invariant to each column's sign:
  L = sum_j (1 - (z_j . u_j)^2 / |z_j|^2)
Subspace form, against an orthonormal target basis U (n x t), invariant to any rotation of U:
  L = sum_j (1 - |U^T z_j|^2 / |z_j|^2)    (the part of each output column outside span(U))
Span form (b <= t), invariant to rotations of U and to any invertible mixing of Z's columns:
  L = b - tr((Z^T Z)^{-1} Z^T U U^T Z)     (b minus the squared cosines of the principal angles
  between span(Z) and span(U)); b copies of one good direction score no better than one.
"""
from __future__ import annotations

import numpy as np

from . import core, rng

NFEAT = 8
STREAM_PROBE = 6


def _rms(x):
    r = np.sqrt(np.mean(x * x))
    return r if r > 0 else 1.0


def features(rowptr, colidx, seed: int) -> np.ndarray:
    """n x 8 feature matrix (FP64), see the module docstring."""
    n = rowptr.shape[0] - 1
    A = lambda X: core.spmm(rowptr, colidx, X)
    d = A(np.ones((n, 1)))[:, 0]
    ad = A(d[:, None])[:, 0]
    a2d = A(ad[:, None])[:, 0]
    R = rng.normal_block(n, 4, seed, STREAM_PROBE)
    P1 = A(R)
    P2 = A(P1)
    P3 = A(P2)
    P4 = A(P3)
    q2 = np.mean(P2 * P2, axis=1)
    q3 = np.mean(P3 * P3, axis=1)
    q4 = np.mean(P4 * P4, axis=1)
    mq2 = np.mean(q2)
    F = np.empty((n, NFEAT))
    F[:, 0] = np.log1p(d)
    F[:, 1] = d / _rms(d)
    F[:, 2] = ad / _rms(ad)
    F[:, 3] = a2d / _rms(a2d)
    F[:, 4] = q2 / _rms(q2)
    F[:, 5] = q3 / _rms(q3)
    F[:, 6] = q4 / _rms(q4)
    F[:, 7] = np.log1p(q2 / (mq2 if mq2 > 0 else 1.0))
    return F


def param_count(hidden: int, b: int) -> int:
    return NFEAT * hidden + hidden + hidden * hidden + hidden + hidden * b + b


def unpack(p: np.ndarray, hidden: int, b: int):
    H = hidden
    o = 0
    W1 = p[o:o + NFEAT * H].reshape(NFEAT, H); o += NFEAT * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H * b].reshape(H, b); o += H * b
    b3 = p[o:o + b]; o += b
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def init_params(hidden: int, b: int, seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (any initialisation works with the same code)."""
    r = np.random.default_rng(seed)
    parts = [r.standard_normal((NFEAT, hidden)) * np.sqrt(2.0 / NFEAT), np.zeros(hidden),
             r.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden), np.zeros(hidden),
             r.standard_normal((hidden, b)) * np.sqrt(1.0 / hidden), np.zeros(b)]
    return np.concatenate([x.ravel() for x in parts])


def forward(F, p, hidden, b):
    W1, b1, W2, b2, W3, b3 = unpack(p, hidden, b)
    a1 = F @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    Z = h2 @ W3 + b3
    return Z, (a1, h1, a2, h2)


def loss(F, p, hidden, b, U) -> float:
    Z, _ = forward(F, p, hidden, b)
    s = np.sum(Z * U, axis=0)
    q = np.sum(Z * Z, axis=0)
    return float(np.sum(1.0 - s * s / q))


def loss_and_grad(F, p, hidden, b, U):
    """L and dL/dp by the chain rule (backpropagation written out)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, hidden, b)
    Z, (a1, h1, a2, h2) = forward(F, p, hidden, b)
    s = np.sum(Z * U, axis=0)
    q = np.sum(Z * Z, axis=0)
    L = float(np.sum(1.0 - s * s / q))
    # d/dz_j of -(s_j^2 / q_j) = -2 s_j / q_j u_j + 2 s_j^2 / q_j^2 z_j
    dZ = (-2.0 * s / q) * U + (2.0 * s * s / (q * q)) * Z
    dW3 = h2.T @ dZ
    db3 = dZ.sum(axis=0)
    dh2 = (dZ @ W3.T) * (a2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    dW1 = F.T @ dh1
    db1 = dh1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, g


def subspace_loss(F, p, hidden, b, U) -> float:
    Z, _ = forward(F, p, hidden, b)
    S = U.T @ Z
    return float(np.sum(1.0 - np.sum(S * S, axis=0) / np.sum(Z * Z, axis=0)))


def subspace_loss_and_grad(F, p, hidden, b, U):
    """Subspace form of the loss and dL/dp; dL/dz_j = -2 U s_j / q_j + 2 |s_j|^2 / q_j^2 z_j
    with s_j = U^T z_j, q_j = |z_j|^2."""
    W1, b1, W2, b2, W3, b3 = unpack(p, hidden, b)
    Z, (a1, h1, a2, h2) = forward(F, p, hidden, b)
    S = U.T @ Z
    q = np.sum(Z * Z, axis=0)
    P = np.sum(S * S, axis=0)
    L = float(np.sum(1.0 - P / q))
    dZ = U @ (-2.0 * S / q) + (2.0 * P / (q * q)) * Z
    return L, _backprop(F, p, hidden, b, dZ, (a1, h1, a2, h2))


def span_loss(F, p, hidden, b, U) -> float:
    Z, _ = forward(F, p, hidden, b)
    S = U.T @ Z
    M = Z.T @ Z
    return float(b - np.trace(np.linalg.solve(M, S.T @ S)))


def span_loss_and_grad(F, p, hidden, b, U):
    """Span form and dL/dp.  With S = U^T Z, M = Z^T Z, N = S^T S:
    dL/dZ = -2 U S M^{-1} + 2 Z M^{-1} N M^{-1}."""
    Z, acts = forward(F, p, hidden, b)
    S = U.T @ Z
    M = Z.T @ Z
    N = S.T @ S
    Mi = np.linalg.inv(M)
    L = float(b - np.trace(Mi @ N))
    dZ = -2.0 * U @ (S @ Mi) + 2.0 * Z @ (Mi @ N @ Mi)
    return L, _backprop(F, p, hidden, b, dZ, acts)


def _backprop(F, p, hidden, b, dZ, acts):
    W1, b1, W2, b2, W3, b3 = unpack(p, hidden, b)
    a1, h1, a2, h2 = acts
    dW3 = h2.T @ dZ
    db3 = dZ.sum(axis=0)
    dh2 = (dZ @ W3.T) * (a2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    dW1 = F.T @ dh1
    db1 = dh1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba, ICLR 2015), bias-corrected; returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
