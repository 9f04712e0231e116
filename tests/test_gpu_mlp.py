"""GPU parity of the learned-start kernels against oracle/mlp.py.

Bars (the benchmark spec): forward within 1e-5 of the CPU forward (FP32), gradients within 1e-4
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
