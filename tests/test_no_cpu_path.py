"""The Python binding has no CPU path: every entry point, given host tensors (or run where no
CUDA device exists), raises instead of computing a result, and creating a CSR handle without a
device fails with the library's own error."""
import pytest
import torch

import graphgen
import paper_1602_01421_gb300 as fe

F64 = dict(dtype=torch.float64)


def _calls():
    V = torch.zeros(3, 100, 4, **F64)
    W = torch.zeros(100, 4, **F64)
    C = torch.zeros(12, 4, **F64)
    npar = fe.mlp_param_count(32, 4)
    F = torch.zeros(100, 6)
    P = torch.zeros(npar)
    calls = {
        "block_gram": lambda: fe.block_gram(V, W),
        "block_gram_tc": lambda: fe.block_gram(V, W, engine="tc"),
        "block_update": lambda: fe.block_update(V, C, W),
        "block_update_tc": lambda: fe.block_update(V, C, W, engine="tc"),
        "block_update_gram": lambda: fe.block_update_gram(V, C, W),
        "block_combine": lambda: fe.block_combine(V, torch.zeros(12, 8, **F64), 2),
        "block_orth": lambda: fe.block_orth(V, W, 1.0),
        "block_orth_first": lambda: fe.block_orth(None, W, 1.0),
        "mlp_forward": lambda: fe.mlp_forward(F, P, 32, 4),
        "mlp_span_loss_grad": lambda: fe.mlp_span_loss_grad(F, P, 32, 4, torch.zeros(100, 8)),
        "mlp_adam": lambda: fe.mlp_adam(P, P.clone(), P.clone(), P.clone(), 1),
    }
    if not torch.cuda.is_available():                      # takes no tensor: needs the device
        calls["random_normal"] = lambda: fe.random_normal(100, 4, dtype=torch.float64, seed=1)
    return calls


NAMES = ["block_gram", "block_gram_tc", "block_update", "block_update_tc", "block_update_gram",
         "block_combine", "block_orth", "block_orth_first", "mlp_forward", "mlp_span_loss_grad",
         "mlp_adam", "random_normal"]


@pytest.mark.parametrize("name", NAMES)
def test_host_tensors_are_refused(name):
    calls = _calls()
    if name not in calls:
        pytest.skip("a CUDA device is present and the call takes no tensor")
    assert set(calls) <= set(NAMES)
    with pytest.raises((ValueError, RuntimeError)) as e:
        calls[name]()
    msg = str(e.value)
    assert "CUDA" in msg or "NVIDIA" in msg or "GPU" in msg, msg


@pytest.mark.skipif(torch.cuda.is_available(), reason="a CUDA device is present")
def test_handle_creation_needs_a_device():
    g = graphgen.rmat(8, seed=1)
    with pytest.raises(fe.FeError):
        fe.Csr.from_graph(g)
