"""GB300-native FlashEigen hot path (arXiv 1602.01421): SpMM on power-law graphs, the Table 1
tall-and-skinny block operations and a GPU-resident Block Krylov-Schur eigensolver.

The computation lives in libfe.so (CUDA for sm_103a, C ABI in include/fe.h); this package
marshals torch tensors (device memory, streams) into those calls.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import FeError, check, load

__all__ = ["Csr", "spmm", "block_gram", "block_update", "block_update_gram", "block_combine", "block_orth",
           "random_normal", "eigs",
           "spmm_t", "svds",
           "FeError", "load", "library_path"]

library_path = _lib.LIB_PATH


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the library's kernels need a GPU (there is no CPU path)")
    load().fe_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _dt(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return _lib.FE_F32
    if t.dtype == torch.float64:
        return _lib.FE_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dev(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")
    return ctypes.c_void_p(t.data_ptr())


class Csr:
    """Handle of a 0/1 pattern CSR matrix on the device (fe_csr_create_ex)."""

    def __init__(self, rowptr: np.ndarray, colidx: np.ndarray, *, validate: bool = True,
                 check_symmetric: bool = False, device_mem_cap_bytes: int = 0,
                 tail_max: int = 0, hub_min: int = 0, hub_chunk: int = 0, panel_nnz: int = 0,
                 copy_timeout_ms: int = 0, semi_direct: bool = False, transpose: bool = False,
                 index_format: str = "auto", ncols: int = 0, l2_persist: bool = False):
        lib = load()
        self._rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self._colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        self.n = int(self._rowptr.shape[0] - 1)
        o = _lib.CsrOpts()
        lib.fe_csr_opts_default(ctypes.byref(o))
        o.validate = int(validate)
        o.check_symmetric = int(check_symmetric)
        o.device_mem_cap_bytes = int(device_mem_cap_bytes)
        o.tail_max, o.hub_min, o.hub_chunk = int(tail_max), int(hub_min), int(hub_chunk)
        o.panel_nnz, o.copy_timeout_ms = int(panel_nnz), int(copy_timeout_ms)
        o.semi_direct = int(semi_direct)
        o.transpose = int(transpose)
        o.index_format = _lib.INDEX_FORMAT[index_format]
        o.ncols = int(ncols)
        o.l2_persist = int(l2_persist)
        h = ctypes.c_void_p()
        check(lib.fe_csr_create_ex(self.n, self._rowptr.ctypes.data_as(ctypes.c_void_p),
                                   self._colidx.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._rowptr = self._colidx = None  # the library keeps its own copy

    @classmethod
    def from_graph(cls, g, **kw):
        """Handle of graph g's adjacency pattern; a directed graph also gets A^T (for spmm_t
        and svds) unless `transpose` is given."""
        kw.setdefault("transpose", bool(getattr(g, "directed", False)))
        return cls(g.rowptr, g.colidx, **kw)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("handle destroyed")
        return self._h

    def info(self) -> dict:
        i = _lib.CsrInfo()
        check(load().fe_csr_get_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _lib.CsrInfo._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().fe_csr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def spmm(h: Csr, X, Y=None):
    """Y = A X (fe_spmm); X (ncols, b), Y (n, b) row-major CUDA tensors, float32 or float64."""
    torch = _torch()
    if Y is None:
        Y = torch.empty((h.n,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
    b = 1 if X.dim() == 1 else X.shape[1]
    _stream()
    check(load().fe_spmm(h.handle, _dev(X, "X"), _dev(Y, "Y"), b, _dt(X)))
    return Y


def spmm_t(h: Csr, X, Y=None):
    """Y = A^T X (fe_spmm_t); the handle needs transpose=True."""
    torch = _torch()
    if Y is None:
        Y = torch.empty_like(X)
    b = 1 if X.dim() == 1 else X.shape[1]
    _stream()
    check(load().fe_spmm_t(h.handle, _dev(X, "X"), _dev(Y, "Y"), b, _dt(X)))
    return Y


def block_gram(V, W, alpha: float = 1.0, G=None, engine: str = "auto"):
    """G = alpha V^T W (fe_block_gram_ex).  V: (nv, n, bv) blocks; W: (n, bw).  G: float64.
    engine: "auto" (tensor cores for supported FP64 shapes), "fma" or "tc"."""
    torch = _torch()
    nv, n, bv = V.shape
    bw = W.shape[1]
    if G is None:
        G = torch.empty((nv * bv, bw), dtype=torch.float64, device=W.device)
    _stream()
    check(load().fe_block_gram_ex(_dev(V, "V"), n, nv, bv, _dev(W, "W"), bw, _dt(W), float(alpha),
                                  _dev(G, "G"), _lib.ENGINE[engine]))
    return G


def block_combine(V, Y, nout: int, Out=None, engine: str = "auto"):
    """Out blocks o = sum_j V_j Y[j-block rows, o-block columns] (fe_block_combine).
    V: (nv, n, bv) blocks; Y: float64 (nv*bv, nout*bv); returns Out (nout, n, bv).
    engine: "auto", "fma" or "tc" (tensor-core split products, FP64 only)."""
    torch = _torch()
    nv, n, bv = V.shape
    if Out is None:
        Out = torch.empty((nout, n, bv), dtype=V.dtype, device=V.device)
    Y = Y.to(torch.float64).contiguous()
    _stream()
    check(load().fe_block_combine(_dev(V, "V"), n, nv, bv, _dev(Y, "Y"), nout, _dev(Out, "Out"),
                                  _dt(V), _lib.ENGINE[engine]))
    return Out


def block_update(V, C, W, alpha: float = 1.0, beta: float = 1.0, engine: str = "fma"):
    """W = beta W + alpha V C (fe_block_update_ex).  V: (nv, n, bv) or None; C: float64.
    engine: "fma" (FMA kernels), "auto" or "tc" (tensor-core split products for FP64, bv == bw)."""
    n, bw = W.shape
    if V is None:
        nv, bv, vp, cp = 0, bw, None, None
    else:
        nv, _, bv = V.shape
        vp, cp = _dev(V, "V"), _dev(C, "C")
    _stream()
    check(load().fe_block_update_ex(vp, n, nv, bv, cp, float(alpha), float(beta), _dev(W, "W"), bw,
                                    _dt(W), _lib.ENGINE[engine]))
    return W


def block_update_gram(V, C, W, alpha: float = 1.0, beta: float = 1.0, G=None):
    """W = beta W + alpha V C, then G = [V; W]^T W (fe_block_update_gram).  V: (nv, n, b) or
    None; C: float64 (nv*b, b); G: float64 ((nv+1)*b, b)."""
    torch = _torch()
    n, b = W.shape
    if V is None:
        nv, vp, cp = 0, None, None
    else:
        nv = V.shape[0]
        vp, cp = _dev(V, "V"), _dev(C, "C")
    if G is None:
        G = torch.empty(((nv + 1) * b, b), dtype=torch.float64, device=W.device)
    _stream()
    check(load().fe_block_update_gram(vp, n, nv, b, cp, float(alpha), float(beta), _dev(W, "W"),
                                      _dt(W), _dev(G, "G")))
    return G


def block_orth(V, W, anorm: float, seed: int = 1):
    """CGS2 + CholeskyQR2 of W against V (fe_block_orth); returns (G, R, replaced)."""
    torch = _torch()
    n, b = W.shape
    nv = 0 if V is None else V.shape[0]
    G = torch.zeros((max(nv, 1) * b, b), dtype=torch.float64, device=W.device)
    R = torch.zeros((b, b), dtype=torch.float64, device=W.device)
    rep = ctypes.c_int(0)
    _stream()
    check(load().fe_block_orth(None if V is None else _dev(V, "V"), n, nv, b, _dev(W, "W"),
                               _dt(W), float(anorm), int(seed), _dev(G, "G"), _dev(R, "R"),
                               ctypes.byref(rep)))
    return G[: nv * b], R, rep.value


def random_normal(n: int, b: int, dtype=None, seed: int = 1, stream: int = 4, offset: int = 0,
                  device="cuda"):
    """MvRandom (fe_random_normal): counter-based N(0,1) row-major (n, b) block."""
    torch = _torch()
    X = torch.empty((n, b), dtype=dtype or torch.float64, device=device)
    _stream()
    check(load().fe_random_normal(_dev(X, "X"), n, b, _dt(X), int(seed), int(stream),
                                  int(offset)))
    return X


def eigs(h: Csr, nev: int, block: int, nblocks: int, tol: float = 1e-8, which: str = "LM", *,
         mode: str = "fp64", start=None, seed: int = 1, max_restarts: int = 500,
         mlp_weights=None, mlp_hidden: int = 64, mixed_tol: float = 5e-6,
         orth_pass1: str = "fp32", return_vectors: bool = True, raise_on_noconverge: bool = True,
         subspace: str = "device", engine: str = "auto", orth_local: bool = True):
    """Block Krylov-Schur (fe_eigs_ex).  subspace="host" keeps the subspace blocks in pinned
    host memory (newest block cached on the device).  Returns (evals numpy, evecs (n, nev) CUDA float64 or
    None, stats dict).  orth_pass1: "fp32" or "fp64" arithmetic for the first Gram-Schmidt
    pass's Gram on an FP64 subspace.  engine: "auto"/"tc" (tensor-core restart products where
    supported) or "fma".  orth_local: first Gram-Schmidt pass from the projected matrix's
    symmetry (only v_j^T W computed) instead of a full Gram."""
    torch = _torch()
    lib = load()
    o = _lib.EigsOpts()
    lib.fe_eigs_opts_default(ctypes.byref(o))
    o.seed = int(seed)
    o.max_restarts = int(max_restarts)
    o.mode = _lib.MODE[mode]
    o.mixed_tol = float(mixed_tol)
    o.orth_pass1 = {"fp32": 0, "fp64": 1}[orth_pass1]
    o.subspace_host = {"device": 0, "host": 1}[subspace]
    o.engine = _lib.ENGINE[engine]
    o.orth_local = 1 if orth_local else 0
    o.mlp_hidden = int(mlp_hidden)
    if start is not None:
        start = start.to(torch.float64).contiguous()
        o.start = _lib.START["user"]
        o.start_block = start.data_ptr()
    elif mlp_weights is not None:
        o.start = _lib.START["learned"]
        o.mlp_weights = mlp_weights.data_ptr()
    evals = np.zeros(nev, dtype=np.float64)
    evecs_cm = torch.empty((nev, h.n), dtype=torch.float64, device="cuda") if return_vectors else None
    st = _lib.EigsStats()
    _stream()
    rc = lib.fe_eigs_ex(h.handle, nev, block, nblocks, float(tol), _lib.WHICH[which],
                        ctypes.byref(o), evals.ctypes.data_as(ctypes.c_void_p),
                        None if evecs_cm is None else ctypes.c_void_p(evecs_cm.data_ptr()),
                        ctypes.byref(st))
    stats = {f: getattr(st, f) for f, _ in _lib.EigsStats._fields_}
    stats["converged"] = rc == _lib.FE_OK
    if rc != _lib.FE_OK and not (rc == _lib.FE_ERR_NOCONVERGE and not raise_on_noconverge):
        check(rc)
    return evals, (None if evecs_cm is None else evecs_cm.t()), stats


def svds(h: Csr, nsv: int, block: int, nblocks: int, tol: float = 1e-8, *, mode: str = "fp64",
         start=None, seed: int = 1, max_restarts: int = 500, mixed_tol: float = 5e-6,
         orth_pass1: str = "fp32", return_vectors: bool = True, raise_on_noconverge: bool = True,
         subspace: str = "device", engine: str = "auto"):
    """Largest singular triplets of the handle's matrix (fe_svds; needs transpose=True).
    Returns (svals numpy, right (n, nsv) CUDA float64 or None, left (n, nsv) or None, stats)."""
    torch = _torch()
    lib = load()
    o = _lib.EigsOpts()
    lib.fe_eigs_opts_default(ctypes.byref(o))
    o.seed = int(seed)
    o.max_restarts = int(max_restarts)
    o.mode = _lib.MODE[mode]
    o.mixed_tol = float(mixed_tol)
    o.orth_pass1 = {"fp32": 0, "fp64": 1}[orth_pass1]
    o.subspace_host = {"device": 0, "host": 1}[subspace]
    o.engine = _lib.ENGINE[engine]
    if start is not None:
        start = start.to(torch.float64).contiguous()
        o.start = _lib.START["user"]
        o.start_block = start.data_ptr()
    svals = np.zeros(nsv, dtype=np.float64)
    right = left = None
    if return_vectors:
        right = torch.empty((nsv, h.n), dtype=torch.float64, device="cuda")
        left = torch.empty((nsv, h.n), dtype=torch.float64, device="cuda")
    st = _lib.EigsStats()
    _stream()
    rc = lib.fe_svds(h.handle, nsv, block, nblocks, float(tol), ctypes.byref(o),
                     svals.ctypes.data_as(ctypes.c_void_p),
                     None if right is None else ctypes.c_void_p(right.data_ptr()),
                     None if left is None else ctypes.c_void_p(left.data_ptr()), ctypes.byref(st))
    stats = {f: getattr(st, f) for f, _ in _lib.EigsStats._fields_}
    stats["converged"] = rc == _lib.FE_OK
    if rc != _lib.FE_OK and not (rc == _lib.FE_ERR_NOCONVERGE and not raise_on_noconverge):
        check(rc)
    return (svals, None if right is None else right.t(), None if left is None else left.t(),
            stats)


# ---------------------------------------------------------------- learned start block
NFEAT = 8


def mlp_param_count(hidden: int, b: int) -> int:
    c = load().fe_mlp_param_count(int(hidden), int(b))
    if c < 0:
        raise ValueError("hidden must be 32 or 64 and b in {1,2,4,8,16}")
    return int(c)


def vertex_features(h: Csr, seed: int = 1):
    """n x 8 FP32 features from SpMM powers (fe_vertex_features)."""
    torch = _torch()
    F = torch.empty((h.n, NFEAT), dtype=torch.float32, device="cuda")
    _stream()
    check(load().fe_vertex_features(h.handle, int(seed), _dev(F, "F")))
    return F


def mlp_forward(F, params, hidden: int, b: int):
    torch = _torch()
    Z = torch.empty((F.shape[0], b), dtype=torch.float32, device=F.device)
    _stream()
    check(load().fe_mlp_forward(_dev(F, "F"), F.shape[0], _dev(params, "params"), hidden, b,
                                _dev(Z, "Z")))
    return Z


def mlp_loss_grad(F, params, hidden: int, b: int, U, grad=None):
    """(loss, grad) of the sign-invariant start-block loss (fe_mlp_loss_grad)."""
    torch = _torch()
    if grad is None:
        grad = torch.empty_like(params)
    loss = ctypes.c_double(0.0)
    _stream()
    check(load().fe_mlp_loss_grad(_dev(F, "F"), F.shape[0], _dev(params, "params"), hidden, b,
                                  _dev(U, "U"), _dev(grad, "grad"), ctypes.byref(loss)))
    return loss.value, grad


def mlp_subspace_loss_grad(F, params, hidden: int, b: int, U, grad=None):
    """(loss, grad) of the rotation-invariant subspace loss against an n x t basis U."""
    torch = _torch()
    if grad is None:
        grad = torch.empty_like(params)
    loss = ctypes.c_double(0.0)
    _stream()
    check(load().fe_mlp_subspace_loss_grad(_dev(F, "F"), F.shape[0], _dev(params, "params"),
                                           hidden, b, _dev(U, "U"), U.shape[1], _dev(grad, "grad"),
                                           ctypes.byref(loss)))
    return loss.value, grad


def mlp_span_loss_grad(F, params, hidden: int, b: int, U, grad=None):
    """(loss, grad) of the span form: b - tr((Z^T Z)^-1 Z^T U U^T Z)."""
    torch = _torch()
    if grad is None:
        grad = torch.empty_like(params)
    loss = ctypes.c_double(0.0)
    _stream()
    check(load().fe_mlp_span_loss_grad(_dev(F, "F"), F.shape[0], _dev(params, "params"), hidden,
                                       b, _dev(U, "U"), U.shape[1], _dev(grad, "grad"),
                                       ctypes.byref(loss)))
    return loss.value, grad


def mlp_adam(params, grad, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9,
             beta2: float = 0.999, eps: float = 1e-8):
    _stream()
    check(load().fe_mlp_adam(_dev(params, "params"), _dev(grad, "grad"), _dev(m, "m"),
                             _dev(v, "v"), params.numel(), lr, beta1, beta2, eps, int(step)))
    return params
