"""ctypes binding of libfe.so (include/fe.h).  Argument marshalling only: every step of the
computation runs in the library's CUDA kernels.  Importing this module never falls back to
anything else: if the library is missing, loading raises."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfe.so")

FE_OK = 0
FE_ERR_INVALID = -1
FE_ERR_OOM = -2
FE_ERR_CUDA = -3
FE_ERR_NOCONVERGE = -4
FE_ERR_TIMEOUT = -5
FE_ERR_DEVICE_CHECK = -6
FE_F32, FE_F64 = 0, 1
WHICH = {"LM": 0, "LA": 1, "SA": 2}
MODE = {"fp64": 0, "mixed": 1}
START = {"random": 0, "user": 1, "learned": 2}
INDEX_FORMAT = {"auto": 0, "plain": 1, "packed": 2}
ENGINE = {"auto": 0, "fma": 1, "tc": 2}


class CsrOpts(ctypes.Structure):
    _fields_ = [("device_mem_cap_bytes", ctypes.c_int64), ("validate", ctypes.c_int),
                ("check_symmetric", ctypes.c_int), ("tail_max", ctypes.c_int),
                ("hub_min", ctypes.c_int), ("hub_chunk", ctypes.c_int),
                ("panel_nnz", ctypes.c_int64), ("copy_timeout_ms", ctypes.c_int),
                ("semi_direct", ctypes.c_int), ("index_format", ctypes.c_int),
                ("transpose", ctypes.c_int), ("ncols", ctypes.c_int64),
                ("l2_persist", ctypes.c_int)]


class CsrInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rows_empty", ctypes.c_int64),
                ("rows_tail", ctypes.c_int64), ("rows_mid", ctypes.c_int64),
                ("rows_hub", ctypes.c_int64), ("hub_chunks", ctypes.c_int64),
                ("max_degree", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("semi_external", ctypes.c_int), ("panels", ctypes.c_int64),
                ("has_transpose", ctypes.c_int), ("tail_max", ctypes.c_int),
                ("index_format", ctypes.c_int), ("index_bytes", ctypes.c_int64),
                ("ncols", ctypes.c_int64)]


class EigsOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("max_restarts", ctypes.c_int), ("mode", ctypes.c_int),
                ("start", ctypes.c_int), ("start_block", ctypes.c_void_p),
                ("mlp_weights", ctypes.c_void_p), ("mlp_hidden", ctypes.c_int),
                ("mixed_tol", ctypes.c_double), ("max_sweeps", ctypes.c_int),
                ("orth_pass1", ctypes.c_int), ("subspace_host", ctypes.c_int),
                ("engine", ctypes.c_int), ("orth_local", ctypes.c_int)]


class EigsStats(ctypes.Structure):
    _fields_ = [("nconv", ctypes.c_int), ("restarts", ctypes.c_int),
                ("spmm_blocks", ctypes.c_int64), ("spmm_blocks_fp32", ctypes.c_int64),
                ("restarts_fp32", ctypes.c_int), ("replacements", ctypes.c_int), ("anorm", ctypes.c_double),
                ("max_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("seconds_fp32", ctypes.c_double), ("spmm_start", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libfe.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError(f"{LIB_PATH} not built")
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "fe_last_error": (ctypes.c_char_p, []),
            "fe_version": (ctypes.c_char_p, []),
            "fe_set_stream": (i32, [vp]),
            "fe_get_stream": (vp, []),
            "fe_csr_opts_default": (None, [ctypes.POINTER(CsrOpts)]),
            "fe_csr_create": (i32, [i64, vp, vp, ctypes.POINTER(vp)]),
            "fe_csr_create_ex": (i32, [i64, vp, vp, ctypes.POINTER(CsrOpts), ctypes.POINTER(vp)]),
            "fe_csr_destroy": (i32, [vp]),
            "fe_csr_get_info": (i32, [vp, ctypes.POINTER(CsrInfo)]),
            "fe_spmm": (i32, [vp, vp, vp, i32, i32]),
            "fe_spmm_t": (i32, [vp, vp, vp, i32, i32]),
            "fe_svds": (i32, [vp, i32, i32, i32, dbl, ctypes.POINTER(EigsOpts), vp, vp, vp,
                              ctypes.POINTER(EigsStats)]),
            "fe_block_gram": (i32, [vp, i64, i32, i32, vp, i32, i32, dbl, vp]),
            "fe_block_update": (i32, [vp, i64, i32, i32, vp, dbl, dbl, vp, i32, i32]),
            "fe_block_update_ex": (i32, [vp, i64, i32, i32, vp, dbl, dbl, vp, i32, i32, i32]),
            "fe_block_combine": (i32, [vp, i64, i32, i32, vp, i32, vp, i32, i32]),
            "fe_block_gram_ex": (i32, [vp, i64, i32, i32, vp, i32, i32, dbl, vp, i32]),
            "fe_partition_rows": (i32, [i64, vp, i32, vp]),
            "fe_partition_local": (i32, [i64, vp, vp, i64, i64, vp, vp, vp, ctypes.POINTER(i64)]),
            "fe_block_update_gram": (i32, [vp, i64, i32, i32, vp, dbl, dbl, vp, i32, vp]),
            "fe_block_orth": (i32, [vp, i64, i32, i32, vp, i32, dbl, ctypes.c_uint64, vp, vp,
                                    ctypes.POINTER(i32)]),
            "fe_random_normal": (i32, [vp, i64, i32, i32, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64]),
            "fe_eigs_opts_default": (None, [ctypes.POINTER(EigsOpts)]),
            "fe_kernel_launches": (ctypes.c_int64, []),
            "fe_mlp_param_count": (ctypes.c_int64, [i32, i32]),
            "fe_vertex_features": (i32, [vp, ctypes.c_uint64, vp]),
            "fe_mlp_forward": (i32, [vp, i64, vp, i32, i32, vp]),
            "fe_mlp_loss_grad": (i32, [vp, i64, vp, i32, i32, vp, vp, ctypes.POINTER(dbl)]),
            "fe_mlp_adam": (i32, [vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, i32]),
            "fe_mlp_subspace_loss_grad": (i32, [vp, i64, vp, i32, i32, vp, i32, vp,
                                                ctypes.POINTER(dbl)]),
            "fe_mlp_span_loss_grad": (i32, [vp, i64, vp, i32, i32, vp, i32, vp,
                                            ctypes.POINTER(dbl)]),
            "fe_block_gram_noalloc": (i32, [vp, i64, i32, i32, vp, i32, i32, dbl, vp]),
            "fe_eigs": (i32, [vp, i32, i32, i32, dbl, i32, vp, vp]),
            "fe_eigs_ex": (i32, [vp, i32, i32, i32, dbl, i32, ctypes.POINTER(EigsOpts), vp, vp,
                                 ctypes.POINTER(EigsStats)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class FeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def check(rc: int) -> int:
    if rc != FE_OK:
        raise FeError(rc, load().fe_last_error().decode(errors="replace"))
    return rc
