"""The seeded input generators (graphgen): determinism, independence from the thread count,
and the structural rules of the R-MAT recipe (symmetric or directed, no self-loops, no
duplicate entries, sorted rows)."""
import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _digest(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.rowptr).tobytes())
    h.update(np.ascontiguousarray(g.colidx).tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("directed", [False, True])
def test_rmat_same_seed_same_graph_other_seed_other_graph(directed):
    a = graphgen.rmat(12, seed=5, directed=directed)
    b = graphgen.rmat(12, seed=5, directed=directed)
    c = graphgen.rmat(12, seed=6, directed=directed)
    assert _digest(a) == _digest(b)
    assert _digest(a) != _digest(c)


def test_rmat_independent_of_thread_count():
    """Edges come from a counter-based hash of (seed, edge, level), so the graph does not depend
    on how OpenMP splits the draws."""
    code = ("import sys; sys.path.insert(0, %r); import graphgen, hashlib, numpy as np; "
            "g = graphgen.rmat(13, seed=9); h = hashlib.sha256(); "
            "h.update(g.rowptr.tobytes()); h.update(g.colidx.tobytes()); print(h.hexdigest())" % ROOT)
    outs = set()
    for threads in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           check=True)
        outs.add(r.stdout.strip())
    outs.add(_digest(graphgen.rmat(13, seed=9)))
    assert len(outs) == 1


@pytest.mark.parametrize("directed", [False, True])
def test_rmat_structure(directed):
    g = graphgen.rmat(11, seed=2, directed=directed)
    n = g.n
    assert n == 2048 and g.rowptr[0] == 0 and np.all(np.diff(g.rowptr) >= 0)
    assert g.colidx.dtype == np.int32 and g.colidx.min() >= 0 and g.colidx.max() < n
    rows = np.repeat(np.arange(n), g.degrees())
    assert not np.any(rows == g.colidx)                       # no self-loops
    for i in range(n):                                        # sorted, no duplicates
        r = g.colidx[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(r) > 0)
    d = g.dense()
    if directed:
        assert np.abs(d - d.T).sum() > 0
    else:
        assert np.array_equal(d, d.T)
    # edge factor 16: at most 16 n draws, each stored once (directed) or twice (symmetrised)
    assert g.nnz <= (1 if directed else 2) * 16 * n


def test_rmat_scale14_recipe_size():
    """The benchmark's small configuration (scale 14, seed 1): the non-zero count that
    the input recipe documents."""
    g = graphgen.rmat(14, seed=1)
    assert g.n == 16384 and g.nnz == 426382


def test_directed_families():
    assert graphgen.directed_cycle(5).nnz == 5
    assert graphgen.out_star(7).nnz == 6 and graphgen.out_star(7).degrees()[0] == 6
    assert graphgen.transitive_tournament(6).nnz == 15
    g = graphgen.complete_bipartite_directed(3, 4)
    assert g.nnz == 12 and np.all(g.degrees()[:3] == 4) and np.all(g.degrees()[3:] == 0)
