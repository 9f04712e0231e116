"""Closed-form adjacency spectra (pins; see tests/golden/closed_form_spectra.txt)."""
import math
import os

import numpy as np

import graphgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "closed_form_spectra.txt")


def spectrum(family: str, size: int) -> np.ndarray:
    if family == "cycle":
        return 2.0 * np.cos(2.0 * np.pi * np.arange(size) / size)
    if family == "complete":
        return np.array([size - 1.0] + [-1.0] * (size - 1))
    if family == "star":
        r = math.sqrt(size - 1)
        return np.array([r, -r] + [0.0] * (size - 2))
    if family == "hypercube":
        return np.concatenate([[size - 2.0 * i] * math.comb(size, i) for i in range(size + 1)])
    if family == "path":
        return 2.0 * np.cos(np.pi * np.arange(1, size + 1) / (size + 1))
    raise ValueError(family)


def graph(family: str, size: int) -> graphgen.CSR:
    return {"cycle": graphgen.cycle, "complete": graphgen.complete, "star": graphgen.star,
            "hypercube": graphgen.hypercube, "path": graphgen.path}[family](size)


def wanted(family: str, size: int, nev: int, which: str) -> np.ndarray:
    lam = spectrum(family, size)
    if which == "LA":
        return np.sort(lam)[::-1][:nev]
    if which == "SA":
        return np.sort(lam)[:nev]
    order = np.lexsort((-lam, -np.abs(lam)))
    return lam[order][:nev]


def cases():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fam, size, nev, block, nblocks, which = line.split()
            out.append((fam, int(size), int(nev), int(block), int(nblocks), which))
    return out
