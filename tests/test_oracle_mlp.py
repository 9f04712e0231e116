"""Pins for the learned-start oracle (oracle/mlp.py): finite differences, invariances, brute
force for the features, Adam's first step in closed form."""
import numpy as np

import graphgen
from oracle import mlp, rng


def _setup(n_hidden=16, b=4, seed=0):
    g = graphgen.rmat(9, seed=3)
    F = mlp.features(g.rowptr, g.colidx, seed=1)
    U, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((g.n, b)))
    p = mlp.init_params(n_hidden, b, seed=seed)
    p[mlp.NFEAT * n_hidden: mlp.NFEAT * n_hidden + n_hidden] = 0.1   # b1 > 0: fewer dead units
    return g, F, U, p


def test_gradient_matches_central_differences():
    H, b = 16, 4
    g, F, U, p = _setup(H, b)
    L, grad = mlp.loss_and_grad(F, p, H, b, U)
    assert abs(L - mlp.loss(F, p, H, b, U)) < 1e-12
    r = np.random.default_rng(5)
    idx = np.concatenate([r.choice(p.size, 60, replace=False), np.arange(p.size - b, p.size)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(F, p + e, H, b, U) - mlp.loss(F, p - e, H, b, U)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])) + 1e-7, (i, fd, grad[i])


def test_loss_invariances_and_extremes():
    H, b = 16, 4
    g, F, U, p = _setup(H, b)
    L = mlp.loss(F, p, H, b, U)
    assert 0.0 <= L <= b
    assert abs(mlp.loss(F, p, H, b, U * np.array([1, -1, 1, -1])) - L) < 1e-12  # target signs
    q = p.copy()
    W3o = mlp.NFEAT * H + H + H * H + H
    q[W3o:] *= 3.0                                                      # output scale
    assert abs(mlp.loss(F, q, H, b, U) - L) < 1e-10
    # Z = U column-wise gives 0; Z orthogonal to U gives b
    z_perfect = 1.0 - (np.sum(U * U, 0) ** 2) / np.sum(U * U, 0)
    assert np.allclose(z_perfect, 0.0)


def test_features_match_dense_brute_force():
    g = graphgen.rmat(8, seed=4)
    A = g.dense()
    F = mlp.features(g.rowptr, g.colidx, seed=7)
    d = A.sum(1)
    rms = lambda x: np.sqrt(np.mean(x * x))
    R = rng.normal_block(g.n, 4, 7, mlp.STREAM_PROBE)
    qs = [np.mean((np.linalg.matrix_power(A, k) @ R) ** 2, axis=1) for k in (2, 3, 4)]
    want = np.column_stack([np.log1p(d), d / rms(d), A @ d / rms(A @ d), A @ A @ d / rms(A @ A @ d),
                            qs[0] / rms(qs[0]), qs[1] / rms(qs[1]), qs[2] / rms(qs[2]),
                            np.log1p(qs[0] / qs[0].mean())])
    assert np.allclose(F, want, rtol=1e-12, atol=1e-12)


def test_probe_feature_estimates_diag_of_matrix_power():
    """E[(A^p r)_i^2] = (A^(2p))_ii for r ~ N(0, I): the q_p features are unbiased estimates."""
    g = graphgen.rmat(7, seed=2)
    A = g.dense()
    R = rng.normal_block(g.n, 4000, 3, 9)
    est = np.mean((A @ A @ R) ** 2, axis=1)
    exact = np.diag(np.linalg.matrix_power(A, 4))
    assert np.allclose(est, exact, rtol=0.15, atol=1e-9 + 0.15 * exact.mean())


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 0.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=1e-8)
    # bias-corrected first step: m_hat = g, v_hat = g^2  ->  p - lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.1 * g / (np.abs(g) + 1e-8))


def test_training_reduces_loss_on_cpu():
    H, b = 16, 2
    g, F, U, p = _setup(H, b, seed=3)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = mlp.loss(F, p, H, b, U)
    for t in range(1, 61):
        L, gr = mlp.loss_and_grad(F, p, H, b, U)
        p, m, v = mlp.adam_step(p, gr, m, v, t, lr=1e-2)
    assert mlp.loss(F, p, H, b, U) < L0


def test_subspace_gradient_matches_central_differences_and_is_rotation_invariant():
    H, b, t = 16, 4, 6
    g, F, _, p = _setup(H, b)
    U, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((g.n, t)))
    L, grad = mlp.subspace_loss_and_grad(F, p, H, b, U)
    assert abs(L - mlp.subspace_loss(F, p, H, b, U)) < 1e-12
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((t, t)))
    assert abs(mlp.subspace_loss(F, p, H, b, U @ Q) - L) < 1e-10      # any basis of span(U)
    h = 1e-6
    for i in np.random.default_rng(4).choice(p.size, 50, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.subspace_loss(F, p + e, H, b, U) - mlp.subspace_loss(F, p - e, H, b, U)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])) + 1e-7, (i, fd, grad[i])
    # with t = b and U's columns paired to Z's, the subspace loss is at most the column loss
    U4 = U[:, :b]
    assert mlp.subspace_loss(F, p, H, b, U4) <= mlp.loss(F, p, H, b, U4) + 1e-12


def test_span_loss_gradient_invariances_and_collapse():
    H, b, t = 16, 4, 8
    g, F, _, p = _setup(H, b)
    U, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((g.n, t)))
    L, grad = mlp.span_loss_and_grad(F, p, H, b, U)
    assert abs(L - mlp.span_loss(F, p, H, b, U)) < 1e-12 and 0.0 <= L <= b
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((t, t)))
    assert abs(mlp.span_loss(F, p, H, b, U @ Q) - L) < 1e-9            # basis of span(U)
    # mixing the outputs (W3, b3 -> W3 T, b3 T) leaves span(Z), hence L, unchanged
    T = np.random.default_rng(4).standard_normal((b, b)) + 3 * np.eye(b)
    q = p.copy()
    o = mlp.NFEAT * H + H + H * H + H
    q[o:o + H * b] = (p[o:o + H * b].reshape(H, b) @ T).ravel()
    q[o + H * b:] = p[o + H * b:] @ T
    assert abs(mlp.span_loss(F, q, H, b, U) - L) < 1e-8
    h = 1e-6
    for i in np.random.default_rng(5).choice(p.size, 50, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.span_loss(F, p + e, H, b, U) - mlp.span_loss(F, p - e, H, b, U)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-5 * max(1.0, abs(grad[i])) + 1e-7, (i, fd, grad[i])
