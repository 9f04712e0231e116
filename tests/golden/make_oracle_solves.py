"""Writes oracle_solves.json: full oracle solves of the benchmark's R-MAT workloads.

Each entry is one run of the CPU oracle's FP64 Block Krylov-Schur (oracle.bks, Algorithm 1
of Section 3.1 in block form) to convergence on a seeded R-MAT graph: 8 largest-magnitude
eigenpairs, block 4, 8 blocks (subspace 32), tol 1e-8, counter-RNG start seed 1.  The block
SpMM count of the full solve is what the benchmark's CPU arm scales a bounded sample by, so
that the sample is extrapolated by the oracle's own work, not by the GPU's.

    python tests/golden/make_oracle_solves.py [scale ...]      (default: 14 22)

Calls only oracle/ (and graphgen/ for the seeded inputs).  Scale 22 takes tens of minutes.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

NEV, BLOCK, NBLOCKS, TOL = 8, 4, 8, 1e-8
OUT = os.path.join(HERE, "oracle_solves.json")


def main(scales):
    import graphgen
    from oracle import bks
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for sc in scales:
        g = graphgen.rmat(sc, seed=1)
        t0 = time.perf_counter()
        r = bks.block_krylov_schur(g.rowptr, g.colidx, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1,
                                   max_restarts=5000)
        t = time.perf_counter() - t0
        data[f"rmat{sc}"] = {
            "scale": sc, "n": int(g.n), "nnz": int(g.nnz), "nev": NEV, "block": BLOCK,
            "nblocks": NBLOCKS, "tol": TOL, "which": "LM", "seed": 1,
            "converged": bool(r.converged), "restarts": int(r.restarts),
            "spmm_blocks": int(r.spmm_blocks), "evals": [float(x) for x in r.evals],
            "max_resid": float(max(r.resid)), "seconds": round(t, 1),
            "cores": os.cpu_count()}
        print(json.dumps(data[f"rmat{sc}"]), flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [14, 22])
