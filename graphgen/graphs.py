"""Graph and dense-block generators (inputs only; see the package docstring)."""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libfegen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C generator (gcc, OpenMP) into graphgen/_build/libfegen.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.fe_gen_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_int, i64p, ctypes.POINTER(i64p),
                                        ctypes.POINTER(i32p), i64p]
            lib.fe_gen_rmat_ex.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_int, i64p, ctypes.POINTER(i64p),
                                           ctypes.POINTER(i32p), i64p]
            for fn in (lib.fe_gen_symmetrize, lib.fe_gen_directed):
                fn.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p,
                               ctypes.POINTER(i64p), ctypes.POINTER(i32p), i64p]
            lib.fe_gen_free.argtypes = [ctypes.c_void_p]
            lib.fe_gen_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_double)]
            _lib = lib
    return _lib


@dataclasses.dataclass
class CSR:
    """Pattern-only (0/1) CSR: rowptr int64[n+1], colidx int32[nnz].  Symmetric unless
    `directed`, in which case row u lists the out-neighbours of u."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    name: str = ""
    directed: bool = False

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def dense(self) -> np.ndarray:
        """Dense 0/1 adjacency (float64); for small graphs only."""
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), self.degrees())
        a[rows, self.colidx] = 1.0
        return a


def _take_csr(n, rp, ci, nnz, name, directed=False):
    lib = _load()
    rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    colidx = (np.ctypeslib.as_array(ci, shape=(max(nnz, 1),))[:nnz].copy()
              if nnz > 0 else np.zeros(0, np.int32))
    lib.fe_gen_free(ctypes.cast(rp, ctypes.c_void_p))
    lib.fe_gen_free(ctypes.cast(ci, ctypes.c_void_p))
    return CSR(n, rowptr, colidx, name, directed)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True, directed: bool = False) -> CSR:
    """R-MAT graph, n = 2**scale, edge_factor*n directed draws, seeded; symmetrised unless
    `directed` (then the draws are out-edges; self-loops and duplicates dropped either way)."""
    lib = _load()
    n = ctypes.c_int64()
    nnz = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    rc = lib.fe_gen_rmat_ex(scale, edge_factor, a, b, c, seed, 1 if permute else 0,
                            1 if directed else 0, ctypes.byref(n), ctypes.byref(rp),
                            ctypes.byref(ci), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"fe_gen_rmat failed ({rc})")
    return _take_csr(n.value, rp, ci, nnz.value,
                     f"rmat{scale}-ef{edge_factor}-s{seed}{'' if permute else '-noperm'}"
                     f"{'-dir' if directed else ''}", directed)


def from_edges(n: int, src, dst, name: str = "", directed: bool = False) -> CSR:
    """Self-loop-free, duplicate-free CSR from a directed edge list: symmetrised, or the
    out-edge pattern if `directed`."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    assert src.shape == dst.shape
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    i32p = ctypes.POINTER(ctypes.c_int32)
    nnz = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    fn = lib.fe_gen_directed if directed else lib.fe_gen_symmetrize
    rc = fn(n, src.size, src.ctypes.data_as(i32p), dst.ctypes.data_as(i32p),
            ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError("edge list -> CSR failed")
    return _take_csr(n, rp, ci, nnz.value, name, directed)


def cycle(n: int) -> CSR:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, f"cycle{n}")


def path(n: int) -> CSR:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, f"path{n}")


def complete(n: int) -> CSR:
    u, v = np.triu_indices(n, 1)
    return from_edges(n, u, v, f"complete{n}")


def star(n: int) -> CSR:
    """Star S_n: vertex 0 joined to vertices 1..n-1."""
    leaves = np.arange(1, n)
    return from_edges(n, np.zeros(n - 1, np.int64), leaves, f"star{n}")


def hypercube(d: int) -> CSR:
    n = 1 << d
    u = np.repeat(np.arange(n), d)
    v = u ^ (1 << np.tile(np.arange(d), n))
    return from_edges(n, u, v, f"hypercube{d}")


def erdos_renyi(n: int, avg_degree: float, seed: int = 1) -> CSR:
    rng = np.random.default_rng(seed)
    m = int(round(avg_degree * n / 2))
    return from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m), f"er{n}-{avg_degree}")


def disjoint_union(*gs: CSR) -> CSR:
    off = 0
    src, dst = [], []
    for g in gs:
        rows = np.repeat(np.arange(g.n), g.degrees())
        src.append(rows + off)
        dst.append(g.colidx.astype(np.int64) + off)
        off += g.n
    return from_edges(off, np.concatenate(src), np.concatenate(dst), "+".join(g.name for g in gs))


def normal_block(n: int, b: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded N(0,1) row-major n x b block (numpy PCG64)."""
    return np.random.default_rng(seed).standard_normal((n, b)).astype(dtype)


def uniform_block(n: int, b: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded U[0,1) row-major n x b block (numpy PCG64)."""
    return np.random.default_rng(seed).random((n, b)).astype(dtype)


# ---- directed graphs (inputs of the SVD path)

def directed_cycle(n: int) -> CSR:
    """i -> i+1 (mod n): a permutation matrix."""
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, f"dcycle{n}", directed=True)


def out_star(n: int) -> CSR:
    """Vertex 0 -> vertices 1..n-1 (one non-zero row)."""
    return from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), f"ostar{n}", directed=True)


def transitive_tournament(n: int) -> CSR:
    """i -> j for every i < j (the strictly upper triangular all-ones matrix)."""
    u, v = np.triu_indices(n, 1)
    return from_edges(n, u, v, f"ttour{n}", directed=True)


def complete_bipartite_directed(p: int, q: int) -> CSR:
    """Every one of vertices 0..p-1 -> every one of vertices p..p+q-1."""
    u = np.repeat(np.arange(p), q)
    v = np.tile(np.arange(p, p + q), p)
    return from_edges(p + q, u, v, f"dbip{p}x{q}", directed=True)
