"""Training and evaluation of the learned start block (the MLP of fe_mlp_*).

Targets are the leading b Ritz vectors (largest magnitude) that the library's own solver
returns on generated R-MAT graphs; the network is trained on the GPU by the library's
forward/backward/Adam kernels.  Python here only orders the calls.
"""
from __future__ import annotations

import time

import numpy as np

from . import (Csr, eigs, mlp_adam, mlp_loss_grad, mlp_param_count, mlp_span_loss_grad,
               mlp_subspace_loss_grad, vertex_features)

NFEAT = 8


def init_params(hidden: int, b: int, seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases (float32, packed like fe_mlp_param_count)."""
    r = np.random.default_rng(seed)
    parts = [r.standard_normal((NFEAT, hidden)) * np.sqrt(2.0 / NFEAT), np.zeros(hidden),
             r.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden), np.zeros(hidden),
             r.standard_normal((hidden, b)) * np.sqrt(1.0 / hidden), np.zeros(b)]
    p = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert p.size == mlp_param_count(hidden, b)
    return p


def make_example(graph, b: int, feature_seed: int = 1, tol: float = 1e-6, nblocks: int = 8,
                 offset: int = 0, block: int = 4):
    """(features, targets) of one graph: targets = Ritz vectors offset .. offset+b-1 in
    largest-magnitude order (FP32), from the library's own solver."""
    import torch
    nev = offset + b
    with Csr.from_graph(graph) as h:
        F = vertex_features(h, feature_seed)
        _, X, _ = eigs(h, nev, block, nblocks, tol, "LM", mode="mixed", seed=feature_seed)
    U = X[:, offset:offset + b].to(torch.float32).contiguous()
    return F, U


def make_subspace_example(graph, nev: int = 8, block: int = 4, feature_seed: int = 1,
                          tol: float = 1e-6, nblocks: int = 8, first: int = 0):
    """(features, targets) with targets = the wanted Ritz vectors first .. nev-1 (an orthonormal
    basis of part of the wanted invariant subspace), for the subspace and span losses."""
    import torch
    with Csr.from_graph(graph) as h:
        F = vertex_features(h, feature_seed)
        _, X, _ = eigs(h, nev, block, nblocks, tol, "LM", mode="mixed", seed=feature_seed)
    return F, X[:, first:nev].to(torch.float32).contiguous()


def train(examples, hidden: int = 64, b: int = 4, steps: int = 400, lr: float = 3e-3,
          seed: int = 0, log_every: int = 0, loss: str = "column"):
    """Adam on the full-batch loss, cycling through the examples.  Returns (params, losses).
    loss = "column" (output j against target j), "subspace" (each output against span(U)) or
    "span" (span(Z) against span(U))."""
    import torch
    p = torch.from_numpy(init_params(hidden, b, seed)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.empty_like(p)
    losses = []
    for t in range(1, steps + 1):
        F, U = examples[(t - 1) % len(examples)]
        if loss == "subspace":
            L, _ = mlp_subspace_loss_grad(F, p, hidden, b, U, g)
        elif loss == "span":
            L, _ = mlp_span_loss_grad(F, p, hidden, b, U, g)
        else:
            L, _ = mlp_loss_grad(F, p, hidden, b, U, g)
        losses.append(L)
        mlp_adam(p, g, m, v, t, lr=lr)
        if log_every and t % log_every == 0:
            print(f"step {t} loss {np.mean(losses[-log_every:]):.4f}", flush=True)
    return p, losses


def evaluate(graph, params, hidden: int, nev: int = 8, block: int = 4, nblocks: int = 8,
             tol: float = 1e-8, seeds=(1, 2, 3), mode: str = "fp64"):
    """SpMM count and time to nev pairs: learned start vs random starts on one graph."""
    import torch
    out = {"random": [], "learned": None}
    with Csr.from_graph(graph) as h:
        for s in seeds:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, _, st = eigs(h, nev, block, nblocks, tol, "LM", seed=s, mode=mode,
                             return_vectors=False)
            torch.cuda.synchronize()
            out["random"].append({"seed": s, "spmm_blocks": st["spmm_blocks"],
                                  "restarts": st["restarts"], "s": time.perf_counter() - t0,
                                  "evals": ev.tolist()})
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, _, st = eigs(h, nev, block, nblocks, tol, "LM", seed=1, mode=mode,
                         mlp_weights=params, mlp_hidden=hidden, return_vectors=False)
        torch.cuda.synchronize()
        out["learned"] = {"spmm_blocks": st["spmm_blocks"], "spmm_start": st["spmm_start"],
                          "restarts": st["restarts"], "s": time.perf_counter() - t0,
                          "evals": ev.tolist()}
    return out
