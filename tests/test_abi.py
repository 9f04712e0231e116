"""C-ABI library: loads, exports every symbol include/fe.h declares, and rejects bad input on
the host (no GPU needed for any of these)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1602_01421_gb300 as fe
from paper_1602_01421_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported():
    lib = fe.load()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in fe.h but not exported"


def test_version_and_error_string():
    lib = fe.load()
    assert b"sm_103a" in lib.fe_version()
    assert lib.fe_last_error() is not None


@pytest.mark.parametrize("rowptr,colidx,msg", [
    ([1, 2, 3], [0, 1, 1], "rowptr[0]"),
    ([0, 2, 1], [0, 1], "decreases"),
    ([0, 1, 2], [0, 5], "out of range"),
    ([0, 1, 2], [0, -1], "out of range"),
])
def test_invalid_csr_rejected_on_host(rowptr, colidx, msg):
    with pytest.raises(fe.FeError) as e:
        fe.Csr(np.array(rowptr), np.array(colidx, dtype=np.int32))
    assert e.value.code == _lib.FE_ERR_INVALID and msg in str(e.value)


def test_asymmetric_pattern_rejected_when_checked():
    with pytest.raises(fe.FeError) as e:
        fe.Csr(np.array([0, 1, 1]), np.array([1], dtype=np.int32), check_symmetric=True)
    assert "not symmetric" in str(e.value)
    with pytest.raises(fe.FeError) as e:
        fe.Csr(np.array([0, 1, 2]), np.array([0, 1], dtype=np.int32), check_symmetric=True)
    assert "self-loop" in str(e.value)


def test_null_and_bad_arguments():
    lib = fe.load()
    assert lib.fe_spmm(None, None, None, 4, 0) == _lib.FE_ERR_INVALID
    assert lib.fe_spmm_t(None, None, None, 4, 0) == _lib.FE_ERR_INVALID
    assert lib.fe_svds(None, 8, 2, 16, 1e-8, None, None, None, None, None) == _lib.FE_ERR_INVALID
    assert lib.fe_eigs(None, 8, 4, 8, 1e-8, 0, None, None) == _lib.FE_ERR_INVALID
    assert lib.fe_block_gram(None, 10, 1, 4, None, 4, 0, 1.0, None) == _lib.FE_ERR_INVALID
    assert lib.fe_block_update(None, 10, 1, 3, None, 1.0, 0.0, ctypes.c_void_p(16), 4, 0) == _lib.FE_ERR_INVALID
    assert lib.fe_random_normal(None, 10, 4, 1, 1, 4, 0) == _lib.FE_ERR_INVALID
    out = ctypes.c_void_p()
    assert lib.fe_csr_create(0, None, None, ctypes.byref(out)) == _lib.FE_ERR_INVALID


def test_unaligned_blocks_rejected_on_host():
    """Block arguments 8 bytes off a 16-byte boundary: FE_ERR_INVALID with an alignment message
    from every block operation, before any device work (the pointers are never touched)."""
    lib = fe.load()
    V, W, O, C = (ctypes.c_void_p(0x100008), ctypes.c_void_p(0x200000), ctypes.c_void_p(0x300008),
                  ctypes.c_void_p(0x400000))
    Va = ctypes.c_void_p(0x100000)
    f64, n = 1, 1024
    calls = [
        lambda: lib.fe_block_gram_ex(V, n, 2, 4, W, 4, f64, 1.0, C, 0),
        lambda: lib.fe_block_gram(Va, n, 2, 4, ctypes.c_void_p(0x200008), 4, f64, 1.0, C),
        lambda: lib.fe_block_gram_noalloc(V, n, 2, 4, W, 4, f64, 1.0, C),
        lambda: lib.fe_block_update_ex(V, n, 2, 4, C, 1.0, 1.0, W, 4, f64, 0),
        lambda: lib.fe_block_update(Va, n, 2, 4, C, 1.0, 1.0, ctypes.c_void_p(0x200008), 4, f64),
        lambda: lib.fe_block_combine(Va, n, 2, 4, C, 2, O, f64, 0),
        lambda: lib.fe_block_update_gram(V, n, 2, 4, C, 1.0, 1.0, W, f64, C),
        lambda: lib.fe_block_orth(Va, n, 2, 4, ctypes.c_void_p(0x200008), f64, 1.0, 1, C, C, None),
    ]
    for call in calls:
        assert call() == _lib.FE_ERR_INVALID
        assert b"16-byte aligned" in lib.fe_last_error()


def test_bad_index_format_rejected_on_host():
    lib = fe.load()
    rowptr = np.array([0, 1, 2], dtype=np.int64)
    colidx = np.array([1, 0], dtype=np.int32)
    o = _lib.CsrOpts()
    lib.fe_csr_opts_default(ctypes.byref(o))
    o.index_format = 7
    out = ctypes.c_void_p()
    rc = lib.fe_csr_create_ex(2, rowptr.ctypes.data_as(ctypes.c_void_p),
                              colidx.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(out))
    assert rc == _lib.FE_ERR_INVALID and b"index_format" in lib.fe_last_error()


def test_struct_layouts_match_header():
    # field offsets the C compiler gives the structs (x86-64 and aarch64 share the LP64 ABI)
    assert ctypes.sizeof(_lib.CsrOpts) == 72
    assert ctypes.sizeof(_lib.CsrInfo) == 120
    assert ctypes.sizeof(_lib.EigsOpts) == 80
    assert ctypes.sizeof(_lib.EigsStats) == 72


def test_struct_field_offsets_match_c_compiler(tmp_path):
    """Every ctypes field sits at the offset gcc gives the same field of include/fe.h."""
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    structs = {"fe_csr_opts": _lib.CsrOpts, "fe_csr_info": _lib.CsrInfo,
               "fe_eigs_opts": _lib.EigsOpts, "fe_eigs_stats": _lib.EigsStats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fe.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_mlp_param_count_matches_the_oracles_packing():
    """fe_mlp_param_count (host) against the oracle's packed layout [W1, b1, W2, b2, W3, b3];
    -1 for unsupported widths."""
    from oracle import mlp
    lib = fe.load()
    for hidden in (32, 64):
        for b in (1, 2, 4, 8, 16):
            assert lib.fe_mlp_param_count(hidden, b) == mlp.param_count(hidden, b) \
                == 8 * hidden + hidden + hidden * hidden + hidden + hidden * b + b
    for hidden, b in ((16, 4), (32, 3), (48, 4), (64, 32)):
        assert lib.fe_mlp_param_count(hidden, b) == -1
