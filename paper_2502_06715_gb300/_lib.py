"""ctypes declarations of the C ABI in include/honeycomb.h and
include/honeycomb_kary.h.

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

HC_MAX_VARS = 8
HC_MAX_ATOMS = 12
HC_KMAX_ARITY = 3
HC_KMAX_VARS = 6

HC_MODE_COUNT = 0
HC_MODE_MATERIALIZE = 1
HC_FLAG_CELL_COUNTS = 1
HC_FLAG_STATS = 2
HC_FLAG_TIME_KERNELS = 4
HC_FLAG_NO_LIFT = 8
HC_FLAG_CELL_PROFILE = 16
HC_BUILD_CHECK_DUPLICATES = 1
HC_BUILD_TIME_KERNELS = 2
HC_BUILD_TEST_STALL_SORT = 0x100
HC_BUILD_TEST_STALL_SCAN = 0x200

STATUS = {0: "HC_OK", 1: "HC_ERR_ARG", 2: "HC_ERR_OOM", 3: "HC_ERR_CUDA", 4: "HC_ERR_TIMEOUT",
          5: "HC_ERR_CAPACITY", 6: "HC_ERR_DUPLICATE", 7: "HC_ERR_BUSY"}


class hc_atom(ctypes.Structure):
    _fields_ = [("var0", ctypes.c_uint8), ("var1", ctypes.c_uint8)]


class hc_query(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_uint32), ("n_atoms", ctypes.c_uint32),
                ("atoms", hc_atom * HC_MAX_ATOMS), ("order", ctypes.c_uint8 * HC_MAX_VARS)]


class hc_index_view(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("l1", ctypes.c_uint64), ("attr_order", ctypes.c_uint32),
                ("max_first", ctypes.c_uint32), ("max_second", ctypes.c_uint32),
                ("d_v1", ctypes.c_void_p), ("d_o1", ctypes.c_void_p), ("d_v2", ctypes.c_void_p),
                ("d_keys", ctypes.c_void_p), ("ms_radix_passes", ctypes.c_float),
                ("n_radix_passes", ctypes.c_uint32), ("ms_boundary", ctypes.c_float), ("max_run", ctypes.c_uint64),
                ("v1pos_n", ctypes.c_uint32)]


class hc_partitioned_view(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("l1", ctypes.c_uint64), ("n_parts", ctypes.c_uint64),
                ("pa", ctypes.c_uint32), ("pb", ctypes.c_uint32), ("d_keys", ctypes.c_void_p),
                ("d_bpref", ctypes.c_void_p), ("d_v1", ctypes.c_void_p), ("d_o1", ctypes.c_void_p),
                ("d_v2", ctypes.c_void_p), ("d_lvl1_start", ctypes.c_void_p)]


class hc_join_params(ctypes.Structure):
    _fields_ = [("shares", ctypes.c_uint32 * HC_MAX_VARS), ("seeds", ctypes.c_uint32 * HC_MAX_VARS),
                ("mode", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("item_grain", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("merge_min", ctypes.c_uint32), ("merge_ratio", ctypes.c_uint32),
                ("slice_grain", ctypes.c_uint32), ("lift_arena", ctypes.c_uint32), ("out_capacity", ctypes.c_uint64),
                ("dir_min", ctypes.c_uint32), ("pair_min", ctypes.c_uint32)]


class hc_result_view(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("n_tuples", ctypes.c_uint64), ("d_tuples", ctypes.c_void_p),
                ("n_cells", ctypes.c_uint64), ("d_cell_counts", ctypes.c_void_p), ("work", ctypes.c_uint64),
                ("n_items", ctypes.c_uint64), ("ms_join_kernel", ctypes.c_float),
                ("n_join_launches", ctypes.c_uint32), ("d_cell_profile", ctypes.c_void_p)]


class hc_kindex_view(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("arity", ctypes.c_uint32), ("level_cols", ctypes.c_uint8 * HC_KMAX_ARITY),
                ("packed", ctypes.c_uint8), ("len", ctypes.c_uint64 * HC_KMAX_ARITY),
                ("max_value", ctypes.c_uint32 * HC_KMAX_ARITY), ("d_v", ctypes.c_void_p * HC_KMAX_ARITY),
                ("d_o", ctypes.c_void_p * HC_KMAX_ARITY), ("ms_sort", ctypes.c_float), ("ms_levels", ctypes.c_float),
                ("n_parts", ctypes.c_uint32), ("shares", ctypes.c_uint32 * HC_KMAX_ARITY),
                ("seeds", ctypes.c_uint32 * HC_KMAX_ARITY), ("d_bpref", ctypes.c_void_p),
                ("d_level0_start", ctypes.c_void_p)]


class hc_katom(ctypes.Structure):
    _fields_ = [("arity", ctypes.c_uint8), ("var", ctypes.c_uint8 * HC_KMAX_ARITY)]


class hc_kquery(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_uint32), ("n_atoms", ctypes.c_uint32),
                ("atoms", hc_katom * HC_MAX_ATOMS), ("order", ctypes.c_uint8 * HC_MAX_VARS)]


class hc_kjoin_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("item_grain", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("pair_min", ctypes.c_uint32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "hc_build_index": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hc_index_from_stats": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]),
    "hc_set_wait_limit_ns": (ctypes.c_int, [ctypes.c_uint64]),
    "hc_run_join_to_host": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(hc_join_params), ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]),
    "hc_wait_limit_ns": (ctypes.c_uint64, []),
    "hc_build_unary_index": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "hc_index_free": (ctypes.c_int, [ctypes.c_void_p]),
    "hc_coco_levels_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "hc_index_get_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hc_index_view)]),
    "hc_partition_index": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hc_partitioned_get_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hc_partitioned_view)]),
    "hc_partitioned_free": (ctypes.c_int, [ctypes.c_void_p]),
    "hc_choose_shares": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "hc_choose_plan": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32,
                                      ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint32)]),
    "hc_plan_cost": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "hc_run_join": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p),
                                   ctypes.POINTER(hc_join_params), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "hc_result_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hc_result_view)]),
    "hc_join_footprint": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(hc_join_params), ctypes.POINTER(ctypes.c_uint64)]),
    "hc_result_free": (ctypes.c_int, [ctypes.c_void_p]),
    "hc_batch_create": (ctypes.c_int, [ctypes.POINTER(hc_query), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(hc_join_params), ctypes.c_uint32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "hc_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hc_batch_capture": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hc_batch_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "hc_batch_free": (ctypes.c_int, [ctypes.c_void_p]),
    "hc_build_kindex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "hc_build_kindex_partitioned": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                                   ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint32),
                                                   ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "hc_kindex_free": (ctypes.c_int, [ctypes.c_void_p]),
    "hc_kindex_get_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hc_kindex_view)]),
    "hc_run_kjoin": (ctypes.c_int, [ctypes.POINTER(hc_kquery), ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(hc_kjoin_params), ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]),
    "hc_kindex_from_stats": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint8),
                                            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "hc_kplan_cost": (ctypes.c_int, [ctypes.POINTER(hc_kquery), ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "hc_choose_korder": (ctypes.c_int, [ctypes.POINTER(hc_kquery), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_uint8)]),
    "hc_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "hc_last_error": (ctypes.c_char_p, []),
    "hc_version": (ctypes.c_uint32, []),
    "hc_target_sm": (ctypes.c_uint32, []),
    "hc_kernel_launches": (ctypes.c_uint64, []),
}

_LIB = None


class HoneycombError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load the built library (raises if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library is not built ({path}); run "
                           "paper_2502_06715_gb300.build.build_library() or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, where: str) -> None:
    if status != 0:
        lib = load()
        raise HoneycombError(status, where, lib.hc_last_error().decode(errors="replace"))
