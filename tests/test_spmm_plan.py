"""Host logic of the SpMM plan (the degree binning of Section 3.3.3's load balancing, built once
per handle on the host), checked bit for bit on the CPU: the library's own plan builder is run
through a small host-only driver (tests/plan_dump.cu, linked against libfe.so) and every field
of its plan is compared with what the CSR fixes:

* every row of the range appears exactly once -- in the slice bucket of its degree (rows of
  degree <= tail_max, buckets by descending degree, rows in order, 32 per slice, -1 padding),
  as one warp task (tail_max < degree <= hub_min, tasks by descending degree, stable), or as
  hub_chunk-sized chunk tasks (degree > hub_min, first among the tasks, in row order);
* the slices' transposed ELL entries are the rows' columns in CSR order (0 in padding lanes);
* plain tasks point at the row's columns in CSR order; packed tasks decode -- the kernel's
  arithmetic restated: w-bit gap fields LSB first from word woff, c_k = base + g_0 + .. + g_k
  with g_0 = 0, read through a two-word window -- to the sorted columns of the row or chunk,
  with contiguous word-aligned segments and two zero words at the end.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import graphgen
import paper_1602_01421_gb300 as fe
from paper_1602_01421_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    fe.load()                                              # builds libfe.so if it is absent
    libdir = os.path.dirname(_lib.LIB_PATH)
    exe = str(tmp_path_factory.mktemp("plan") / "plan_dump")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1602_01421_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "plan_dump.cu"), "-o", exe, "-L", libdir, "-lfe",
                    "-Xlinker", "-rpath," + libdir], check=True, capture_output=True)
    return exe


class _Reader:
    def __init__(self, data):
        self.b, self.o = data, 0

    def take(self, dtype, count):
        a = np.frombuffer(self.b, dtype=dtype, count=count, offset=self.o)
        self.o += a.nbytes
        return a

    def arr(self, dtype):
        return self.take(dtype, int(self.take(np.int64, 1)[0]))


def build_plan(exe, tmp_path, rowptr, colidx, r0, r1, tail_max, hub_min, hub_chunk, packed):
    n = len(rowptr) - 1
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(src, "wb") as f:
        f.write(np.array([n, r0, r1], dtype=np.int64).tobytes())
        f.write(np.array([tail_max, hub_min, hub_chunk, int(packed)], dtype=np.int32).tobytes())
        f.write(np.asarray(rowptr, dtype=np.int64).tobytes())
        f.write(np.asarray(colidx, dtype=np.int32).tobytes())
    subprocess.run([exe, str(src), str(dst)], check=True, timeout=300)
    r = _Reader(open(dst, "rb").read())
    rc = int(r.take(np.int32, 1)[0])
    assert rc == 0
    keys = ["max_degree", "rows_empty", "rows_tail", "rows_mid", "rows_hub", "nbuckets", "nslices",
            "ell_total", "ntasks", "nhub_tasks", "nhub", "packed"]
    p = dict(zip(keys, (int(x) for x in r.take(np.int64, 12))))
    for k, dt in (("deg_of_bucket", np.int32), ("deg_slice_begin", np.int32),
                  ("deg_ell_base", np.int64), ("slice_rows", np.int32), ("ell", np.int32),
                  ("hub_rows", np.int32), ("hub_task_begin", np.int32)):
        p[k] = r.arr(dt)
    if p["packed"]:
        p["ptasks"] = r.arr(np.int64).reshape(-1, 5)
        p["tbits"] = r.arr(np.uint32)
    else:
        p["tasks"] = r.arr(np.int64).reshape(-1, 3)
        p["tcol"] = r.arr(np.int32)
    assert r.o == len(r.b)
    return p


def decode_packed(tbits, woff, length, base, w):
    """Columns of one packed task, as the SpMM kernel decodes them."""
    mask = (1 << w) - 1
    cols, acc = [], base
    for k in range(length):
        bit = k * w
        wi = woff + (bit >> 5)
        window = int(tbits[wi]) | (int(tbits[wi + 1]) << 32)
        g = (window >> (bit & 31)) & mask
        if k == 0:
            assert g == 0                                  # g_0 = 0: c_0 is the task's base
        acc += g
        cols.append(acc)
    return cols


def expected_tasks(rowptr, colidx, r0, r1, tail_max, hub_min, hub_chunk, packed):
    """(row, columns) of every warp task in plan order."""
    hub, mid = [], []
    for i in range(r0, r1):
        cols = list(colidx[rowptr[i]:rowptr[i + 1]])
        d = len(cols)
        if d <= tail_max:
            continue
        if packed:
            cols = sorted(cols)
        if d > hub_min:
            hub += [(i, cols[c:c + hub_chunk]) for c in range(0, d, hub_chunk)]
        else:
            mid.append((i, cols))
    mid.sort(key=lambda t: -len(t[1]))                     # stable: row order within a degree
    return hub, mid


def check_plan(p, rowptr, colidx, r0, r1, tail_max, hub_min, hub_chunk, packed):
    deg = np.diff(np.asarray(rowptr, dtype=np.int64))[r0:r1]
    rows = np.arange(r0, r1)
    assert p["max_degree"] == (int(deg.max()) if len(deg) else 0)
    assert p["rows_empty"] == int((deg == 0).sum())
    assert p["rows_tail"] == int(((deg >= 1) & (deg <= tail_max)).sum())
    assert p["rows_mid"] == int(((deg > tail_max) & (deg <= hub_min)).sum())
    assert p["rows_hub"] == int((deg > hub_min).sum()) == p["nhub"]
    # slice buckets
    tail_degs = sorted({int(d) for d in deg if d <= tail_max}, reverse=True)
    assert list(p["deg_of_bucket"]) == tail_degs
    slice_rows, ell, sbeg, ebase = [], [], [], []
    for d in tail_degs:
        r = rows[deg == d]
        sbeg.append(len(slice_rows) // 32)
        ebase.append(len(ell))
        nsl = -(-len(r) // 32)
        padded = np.full(nsl * 32, -1, dtype=np.int64)
        padded[:len(r)] = r
        slice_rows += list(padded)
        for sl in range(nsl):
            block = np.zeros((d, 32), dtype=np.int64)       # [t][lane]
            for lane in range(32):
                row = padded[sl * 32 + lane]
                if row >= 0:
                    block[:, lane] = colidx[rowptr[row]:rowptr[row + 1]]
            ell += list(block.ravel())
    assert p["nslices"] == len(slice_rows) // 32 and p["ell_total"] == len(ell)
    assert list(p["deg_slice_begin"]) == sbeg and list(p["deg_ell_base"]) == ebase
    assert np.array_equal(p["slice_rows"], np.asarray(slice_rows, dtype=np.int32))
    assert np.array_equal(p["ell"][:len(ell)], np.asarray(ell, dtype=np.int32))
    # warp tasks: hub chunks first, then mid rows
    hub, mid = expected_tasks(rowptr, colidx, r0, r1, tail_max, hub_min, hub_chunk, packed)
    tasks = hub + mid
    assert p["ntasks"] == len(tasks) and p["nhub_tasks"] == len(hub)
    hub_rows = sorted({r for r, _ in hub})
    assert list(p["hub_rows"]) == hub_rows
    begin = [0]
    for hr in hub_rows:
        begin.append(begin[-1] + sum(1 for r, _ in hub if r == hr))
    assert list(p["hub_task_begin"]) == begin
    if not packed:
        for (row, cols), (start, trow, tlen) in zip(tasks, p["tasks"]):
            assert (trow, tlen) == (row, len(cols))
            assert list(p["tcol"][start:start + tlen]) == cols
    else:
        tb = p["tbits"]
        woff_next = 0
        for (row, cols), (woff, trow, tlen, base, w) in zip(tasks, p["ptasks"]):
            assert (trow, tlen) == (row, len(cols)) and 1 <= w <= 31
            assert woff == woff_next                        # contiguous, word-aligned segments
            woff_next = woff + -(-tlen * w // 32)
            assert base == cols[0]
            assert decode_packed(tb, int(woff), int(tlen), int(base), int(w)) == cols
        assert len(tb) == woff_next + 2 and tb[-1] == 0 and tb[-2] == 0


def _unsorted_with_duplicates(seed):
    """A CSR whose rows are unsorted and repeat columns, with empty rows and one hub."""
    rng = np.random.default_rng(seed)
    n = 3000
    deg = rng.integers(0, 40, n)
    deg[rng.integers(0, n, 200)] = 0
    deg[17] = 2500
    deg[1234] = 700
    rowptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    colidx = rng.integers(0, n, rowptr[-1]).astype(np.int32)
    colidx[rowptr[5]:rowptr[5] + 3] = 7                     # duplicates
    return rowptr, colidx


def _csr(g):
    return g.rowptr, g.colidx


GRAPHS = {"rmat12": lambda: _csr(graphgen.rmat(12, seed=3)),
          "star9000": lambda: _csr(graphgen.star(9000)),
          "cycle1001": lambda: _csr(graphgen.cycle(1001)),
          "complete70": lambda: _csr(graphgen.complete(70)),
          "unsorted_dup": lambda: _unsorted_with_duplicates(4)}
_made = {}


def _graph(name):
    if name not in _made:
        _made[name] = GRAPHS[name]()
    return _made[name]
# (tail_max, hub_min, hub_chunk): the defaults, the packed default tail, and tiny thresholds that
# send rows of every graph down every path
PARAMS = [(128, 4096, 4096), (16, 4096, 4096), (8, 64, 32), (0, 16, 7)]


@pytest.mark.parametrize("packed", [False, True])
@pytest.mark.parametrize("params", PARAMS)
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_plan_matches_csr(dump_exe, tmp_path, name, params, packed):
    rowptr, colidx = _graph(name)
    n = len(rowptr) - 1
    for r0, r1 in ((0, n), (n // 3, n - n // 5)):          # whole matrix and a row panel
        p = build_plan(dump_exe, tmp_path, rowptr, colidx, r0, r1, *params, packed)
        check_plan(p, rowptr, colidx, r0, r1, *params, packed)


def test_plan_check_is_sensitive(dump_exe, tmp_path):
    """A plan with one ELL entry or one gap bit changed fails the checks."""
    rowptr, colidx = _graph("rmat12")
    n = len(rowptr) - 1
    p = build_plan(dump_exe, tmp_path, rowptr, colidx, 0, n, 8, 64, 32, False)
    p["ell"] = p["ell"].copy()
    p["ell"][5] ^= 1
    with pytest.raises(AssertionError):
        check_plan(p, rowptr, colidx, 0, n, 8, 64, 32, False)
    q = build_plan(dump_exe, tmp_path, rowptr, colidx, 0, n, 8, 64, 32, True)
    q["tbits"] = q["tbits"].copy()
    q["tbits"][3] ^= 1 << 9
    with pytest.raises(AssertionError):
        check_plan(q, rowptr, colidx, 0, n, 8, 64, 32, True)
