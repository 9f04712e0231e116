"""GPU parity of the learned-start kernels against oracle/mlp.py.

Bars: forward within 1e-5 of the CPU forward (FP32), gradients within 1e-4
relative; features within FP32 rounding of the FP64 oracle features.
"""
import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from oracle import mlp as omlp
from paper_1602_01421_gb300 import learned
from tests.gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    g = graphgen.rmat(12, seed=8)
    with fe.Csr.from_graph(g) as h:
        F = fe.vertex_features(h, seed=3)
    return g, F


def test_features_match_oracle(small):
    g, F = small
    ref = omlp.features(g.rowptr, g.colidx, seed=3)
    got = F.cpu().numpy().astype(np.float64)
    assert np.allclose(got, ref, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("hidden,b", [(64, 4), (64, 8), (32, 1), (32, 16), (64, 16)])
def test_forward_matches_oracle(small, hidden, b):
    g, F = small
    p = learned.init_params(hidden, b, seed=hidden + b)
    p[omlp.NFEAT * hidden: omlp.NFEAT * hidden + hidden] = 0.05
    Z = fe.mlp_forward(F, to_dev(p), hidden, b).cpu().numpy()
    Zo, _ = omlp.forward(F.cpu().numpy().astype(np.float64), p.astype(np.float64), hidden, b)
    assert np.allclose(Z, Zo, rtol=1e-5, atol=1e-5 * np.abs(Zo).max())


@pytest.mark.parametrize("hidden,b", [(64, 4), (32, 2), (64, 8)])
def test_loss_and_gradient_match_oracle(small, hidden, b):
    g, F = small
    t = torch()
    p = learned.init_params(hidden, b, seed=7)
    p[omlp.NFEAT * hidden: omlp.NFEAT * hidden + hidden] = 0.05
    U, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((g.n, b)))
    L, grad = fe.mlp_loss_grad(F, to_dev(p), hidden, b, to_dev(U, t.float32))
    F64 = F.cpu().numpy().astype(np.float64)
    Lo, go = omlp.loss_and_grad(F64, p.astype(np.float64), hidden, b,
                                U.astype(np.float32).astype(np.float64))
    grad = grad.cpu().numpy().astype(np.float64)
    assert abs(L - Lo) <= 1e-5 * max(1.0, abs(Lo))
    assert np.linalg.norm(grad - go) <= 1e-4 * np.linalg.norm(go)
    assert np.all(np.abs(grad - go) <= 1e-4 * np.abs(go).max())


@pytest.mark.parametrize("b,t", [(4, 8), (4, 4), (8, 8), (4, 16)])
def test_subspace_loss_and_gradient_match_oracle(small, b, t):
    g, F = small
    t_ = torch()
    p = learned.init_params(64, b, seed=11)
    p[omlp.NFEAT * 64: omlp.NFEAT * 64 + 64] = 0.05
    U, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((g.n, t)))
    L, grad = fe.mlp_subspace_loss_grad(F, to_dev(p), 64, b, to_dev(U, t_.float32))
    F64 = F.cpu().numpy().astype(np.float64)
    Lo, go = omlp.subspace_loss_and_grad(F64, p.astype(np.float64), 64, b,
                                         U.astype(np.float32).astype(np.float64))
    grad = grad.cpu().numpy().astype(np.float64)
    assert abs(L - Lo) <= 1e-5 * max(1.0, abs(Lo))
    assert np.linalg.norm(grad - go) <= 1e-4 * np.linalg.norm(go)
    assert np.all(np.abs(grad - go) <= 1e-4 * np.abs(go).max())


@pytest.mark.parametrize("b,t", [(4, 8), (4, 4), (8, 8)])
def test_span_loss_and_gradient_match_oracle(small, b, t):
    g, F = small
    t_ = torch()
    p = learned.init_params(64, b, seed=13)
    p[omlp.NFEAT * 64: omlp.NFEAT * 64 + 64] = 0.05
    U, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((g.n, t)))
    L, grad = fe.mlp_span_loss_grad(F, to_dev(p), 64, b, to_dev(U, t_.float32))
    F64 = F.cpu().numpy().astype(np.float64)
    Lo, go = omlp.span_loss_and_grad(F64, p.astype(np.float64), 64, b,
                                     U.astype(np.float32).astype(np.float64))
    grad = grad.cpu().numpy().astype(np.float64)
    assert abs(L - Lo) <= 1e-5 * max(1.0, abs(Lo))
    assert np.linalg.norm(grad - go) <= 1e-4 * np.linalg.norm(go)


def test_adam_matches_oracle():
    t = torch()
    r = np.random.default_rng(1)
    p = r.standard_normal(1000).astype(np.float32)
    g = r.standard_normal(1000).astype(np.float32)
    pd, gd = to_dev(p), to_dev(g)
    m, v = t.zeros_like(pd), t.zeros_like(pd)
    po, mo, vo = p.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in (1, 2, 3):
        fe.mlp_adam(pd, gd, m, v, step, lr=0.01)
        po, mo, vo = omlp.adam_step(po, g.astype(np.float64), mo, vo, step, lr=0.01)
    assert np.allclose(pd.cpu().numpy(), po, rtol=1e-5, atol=1e-6)


def test_learned_start_solve_is_correct():
    """Any start block must give the same eigenpairs: learned start vs random start."""
    g = graphgen.rmat(13, seed=4)
    p = to_dev(learned.init_params(64, 4, seed=1))
    with fe.Csr.from_graph(g) as h:
        ev0, _, st0 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1)
        ev1, X1, st1 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1, mlp_weights=p, mlp_hidden=64)
    assert st1["converged"] and st1["spmm_start"] == 7
    assert np.allclose(ev1, ev0, rtol=1e-8)


def test_learned_start_with_mixed_precision():
    """The learned start feeds the FP32 phase of the mixed iteration; the FP64 phase then
    reaches the same eigenpairs as the plain FP64 solve from a random start."""
    g = graphgen.rmat(13, seed=4)
    p = to_dev(learned.init_params(64, 4, seed=1))
    with fe.Csr.from_graph(g) as h:
        ev0, _, st0 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1)
        ev1, X1, st1 = fe.eigs(h, 8, 4, 8, 1e-8, "LM", seed=1, mlp_weights=p, mlp_hidden=64,
                               mode="mixed")
    assert st1["converged"] and st1["spmm_start"] == 7 and st1["spmm_blocks_fp32"] > 0
    assert np.allclose(ev1, ev0, rtol=1e-8)
    X = X1.cpu().numpy()
    assert np.abs(X.T @ X - np.eye(8)).max() < 1e-10


@pytest.mark.slow
def test_trained_network_gain_on_a_fresh_graph():
    """What the trained network gains over the method without it (a random start): trained with
    the span loss on small R-MAT graphs (scales 12-17) against their 8 wanted Ritz vectors, its
    4 output columns on a fresh scale-20 graph lie mostly in that graph's wanted subspace
    (span loss well below the ~4 of random columns), while a random block has almost no
    component there.  The solve from either start gives the same eigenpairs; the block-SpMM
    counts are printed, not asserted: the solve's cost is set by an eigenvalue cluster whose
    vectors the per-vertex network does not capture, so the count is within the random-start
    spread."""
    t = torch()
    specs = [(s, 100 + i) for i, s in enumerate([12, 13, 14, 15, 16, 17] * 3)]
    ex = [learned.make_subspace_example(graphgen.rmat(s, seed=gs)) for s, gs in specs]
    p, losses = learned.train(ex, hidden=64, b=4, steps=1500, lr=2e-3, loss="span")
    assert np.mean(losses[-50:]) < 0.5 * np.mean(losses[:20])
    g = graphgen.rmat(20, seed=997)
    F, U = learned.make_subspace_example(g)
    L_trained, _ = fe.mlp_span_loss_grad(F, p, 64, 4, U)
    p0 = to_dev(learned.init_params(64, 4, seed=0))
    L_untrained, _ = fe.mlp_span_loss_grad(F, p0, 64, 4, U)
    R = fe.random_normal(g.n, 4, dtype=t.float64, seed=3).cpu().numpy()
    Q, _ = np.linalg.qr(R)
    Uh = U.cpu().numpy().astype(np.float64)
    L_random = 4.0 - np.linalg.norm(Uh.T @ Q) ** 2
    print(f"span loss on the fresh graph: trained {L_trained:.3f}, untrained {L_untrained:.3f}, "
          f"random block {L_random:.3f} (max 4)")
    assert L_trained < 1.0 and L_trained < 0.5 * L_untrained and L_random > 3.9
    r = learned.evaluate(g, p, 64, mode="fp64")
    print(f"block SpMMs: random starts {[x['spmm_blocks'] for x in r['random']]}, "
          f"learned start {r['learned']['spmm_blocks']} (+7 feature SpMMs)")
    assert np.allclose(r["learned"]["evals"], r["random"][0]["evals"], rtol=1e-8)
