"""ctypes binding of libust.so: the C ABI of include/ust.h under the same names.

Argument marshalling only; every step of the computation runs in the CUDA
library. There is no CPU fallback: if libust.so cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

UST_OK = 0
UST_EINVAL = -1
UST_ENOTCONNECTED = -2
UST_ENOMEM = -3
UST_ECUDA = -4
UST_ETIMEOUT = -5
UST_ENOTCONVERGED = -6
UST_ESTATE = -7


class ust_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class ust_opts(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("kappa", ctypes.c_double), ("cg_tol", ctypes.c_double),
                ("max_pop_rounds", ctypes.c_int32), ("max_cg_iters", ctypes.c_int32),
                ("skip_validation", ctypes.c_int32), ("graph_id", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("solve_fp64", ctypes.c_int32), ("wilson_blocks", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class ust_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("pivot", ctypes.c_int32),
                ("ecc", ctypes.c_int32), ("trees", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("draws", ctypes.c_int64), ("pop_rounds", ctypes.c_int64),
                ("max_pop_rounds", ctypes.c_int32), ("max_round_pops", ctypes.c_int32),
                ("farness", ctypes.c_int64), ("cg_iters", ctypes.c_int32),
                ("cg_refinements", ctypes.c_int32), ("cg_relres", ctypes.c_double),
                ("sample_ctas", ctypes.c_int32), ("sample_threads", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("bfs_ms", ctypes.c_double), ("sample_ms", ctypes.c_double),
                ("reduce_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("combine_ms", ctypes.c_double),
                ("last_trees", ctypes.c_int64), ("last_draws", ctypes.c_int64),
                ("last_phase_cycles", ctypes.c_int64 * 12)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "_length_") else v
        return out


# name -> (restype, argtypes)
_SIGNATURES = {
    "ust_default_opts": (None, [ctypes.POINTER(ust_opts)]),
    "ust_init": (ctypes.c_int, [ctypes.POINTER(ust_csr), ctypes.c_int32, ctypes.POINTER(ust_opts),
                                ctypes.POINTER(ctypes.c_void_p)]),
    "ust_init_batch": (ctypes.c_int, [ctypes.POINTER(ust_csr), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                      ctypes.POINTER(ust_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "ust_select_pivot": (ctypes.c_int, [ctypes.POINTER(ust_csr), ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "ust_batch_size": (ctypes.c_int32, [ctypes.c_void_p]),
    "ust_batch_offsets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ust_batch_graph_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ust_info)]),
    "ust_reset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "ust_sample_aggregate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64]),
    "ust_set_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "ust_centralities": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int32]),
    "ust_diag": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_int32]),
    "ust_tau": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_double]),
    "ust_num_trees": (ctypes.c_int64, [ctypes.c_void_p]),
    "ust_get_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "ust_track_edges": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "ust_get_edge_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "ust_get_column": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "ust_get_bfs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ust_tree_range_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                             ctypes.c_void_p, ctypes.c_int32]),
    "ust_sample_trees": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "ust_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ust_info)]),
    "ust_tree_counts_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                               ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "ust_probe_random_access": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_double)]),
    "ust_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ust_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ust_free": (None, [ctypes.c_void_p]),
}

EXPORTS = tuple(_SIGNATURES)

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libust.so (building it with nvcc first when it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and not os.path.exists(_build.LIB):
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libust.so is not built; run paper_2006_13679_gb300.build()")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class UstError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{load().ust_strerror(code).decode()}: {msg}")
        self.code = code


def check(rc: int, ctx=None) -> None:
    if rc != UST_OK:
        raise UstError(rc, load().ust_last_error(ctx).decode())


def default_opts() -> ust_opts:
    o = ust_opts()
    load().ust_default_opts(ctypes.byref(o))
    return o
