"""ctypes binding of the qmcfi C ABI (include/qmcfi.h): structures and function prototypes, same names.

Argument marshalling only.  Loading fails loudly when the library has not been built: there is no Python or
CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

from .build import LIB

QMC_OK = 0
QMC_PENDING = 1
QMC_ERR_ARG = -1
QMC_ERR_TABLE = -2
QMC_ERR_UNSUPPORTED = -3
QMC_ERR_KINEMATICS = -4
QMC_ERR_CUDA = -5
QMC_ERR_MEMORY = -6
QMC_ERR_DEFORMATION = -7
QMC_ERR_TIMEOUT = -8
QMC_ERR_CANCELLED = -9
QMC_ERR_NOT_FOUND = -10
QMC_ERR_NO_DEVICE = -11
QMC_ERR_NOT_CONVERGED = -12
QMC_ERR_CODEGEN = -13
QMC_ERR_NONFINITE = -14

QMC_MAX_DIM = 6
QMC_MAX_SLOTS = 5
QMC_MAX_ORDERS = 8
QMC_ISLAND_LEVELS = 6
QMC_ISLAND_BINS = QMC_ISLAND_LEVELS + 1


def island_bin_words(n_slots: int) -> int:
    """doubles per (sector, island bin) of qmc_probe_islands' bins: points, then 4 sums per slot"""
    return 1 + 4 * n_slots
QMC_PREC_FP64 = 0
QMC_PREC_MIXED = 1
QMC_EVAL_AUTO = 0
QMC_EVAL_TABLE = 1
QMC_EVAL_GENERATED = 2


class qmc_lattice(ctypes.Structure):
    _fields_ = [("n", c_int64), ("z", c_uint32 * QMC_MAX_DIM)]


class qmc_info(ctypes.Structure):
    _fields_ = [("n_sectors", c_int32), ("dim", c_int32), ("loops", c_int32), ("n_invariants", c_int32),
                ("order_min", c_int32), ("order_max", c_int32), ("kmax", c_int32), ("n_slots", c_int32),
                ("n_deformed", c_int32), ("n_negative", c_int32), ("max_sigma", c_int32), ("max_terms", c_int32),
                ("pre_low", c_int32), ("n_pre", c_int32), ("pre", c_double * (QMC_MAX_ORDERS + 4)),
                ("packed_bytes", c_int64), ("flops_per_eval", c_double), ("transcendentals_per_eval", c_double)]


class qmc_sector_desc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("sigma", c_int32), ("n_slots", c_int32), ("n_terms", c_int32),
                ("flops", c_double)]


class qmc_pass(ctypes.Structure):
    _fields_ = [("lattice", qmc_lattice), ("n_shifts", c_int32), ("transform_r", c_int32), ("precision", c_int32),
                ("block", c_int32), ("points_per_thread", c_int32), ("grid", c_int32), ("evaluator", c_int32),
                ("reserved", c_int32), ("sector_precision", c_void_p), ("sector_active", c_void_p)]


class qmc_batch_item(ctypes.Structure):
    _fields_ = [("packed_host", c_void_p), ("packed_dev", c_void_p), ("pass_", qmc_pass), ("shifts_dev", c_void_p),
                ("lambda_dev", c_void_p), ("sums_dev", c_void_p), ("fails_dev", c_void_p),
                ("abort_flag", c_void_p)]


class qmc_options(ctypes.Structure):
    _fields_ = [("rel_tol", c_double), ("abs_tol", c_double), ("precision", c_int32), ("n_shifts", c_int32),
                ("seed", c_uint64), ("lambda_", c_double), ("max_halvings", c_int32), ("transform_r", c_int32),
                ("ladder_start", c_int32), ("n_lattices", c_int32), ("lattices", POINTER(qmc_lattice)),
                ("shifts", POINTER(c_double)), ("max_n", c_int64), ("max_seconds", c_double), ("block", c_int32),
                ("points_per_thread", c_int32), ("probe_samples", c_int64), ("fp32_budget", c_double),
                ("evaluator", c_int32), ("lock_step", c_int32)]


class qmc_result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("order_min", c_int32), ("n_orders", c_int32),
                ("value", (c_double * 2) * QMC_MAX_ORDERS), ("error", (c_double * 2) * QMC_MAX_ORDERS),
                ("n_final", c_int64), ("evals", c_int64), ("seconds", c_double), ("kernel_ms", c_double),
                ("passes", c_int32), ("lambda_halvings", c_int32), ("fp64_reruns", c_int32),
                ("sign_failures", c_int32), ("queued_seconds", c_double), ("island_sectors", c_int32),
                ("nonfinite_sectors", c_int32)]


class qmc_serving_stats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("queued", c_int64), ("active", c_int64),
                ("peak_active", c_int64), ("rounds", c_int64), ("batched_passes", c_int64),
                ("device_bytes", c_int64), ("shed", c_int64)]


# name -> (restype, argtypes); every symbol declared in include/qmcfi.h
class qmc_gen_info(ctypes.Structure):
    _fields_ = [("family", c_uint64), ("compile_ms", c_double), ("source_bytes", c_int64), ("cubin_bytes", c_int64),
                ("cached", c_int32), ("reserved", c_int32)]


class qmc_tune_result(ctypes.Structure):
    _fields_ = [("block", c_int32), ("points_per_thread", c_int32), ("ms", ctypes.c_float),
                ("n_candidates", c_int32), ("candidate_block", c_int32 * 16),
                ("candidate_points_per_thread", c_int32 * 16), ("candidate_ms", ctypes.c_float * 16)]


PROTOTYPES = {
    "qmc_strerror": (c_char_p, [c_int]),
    "qmc_version": (c_int, []),
    "qmc_prepare": (c_int, [c_void_p, c_size_t, POINTER(c_double), c_int32, c_int32, c_int32, c_void_p, c_size_t,
                            POINTER(qmc_info)]),
    "qmc_sector_desc_get": (c_int, [c_void_p, c_int32, POINTER(qmc_sector_desc)]),
    "qmc_scratch_bytes": (c_size_t, [c_void_p, POINTER(qmc_pass)]),
    "qmc_eval_sums": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_void_p, c_size_t,
                              c_void_p, c_void_p, c_void_p]),
    "qmc_batch_scratch_bytes": (c_size_t, [c_void_p, c_int32]),
    "qmc_eval_batch": (c_int, [c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "qmc_eval_partials": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_void_p, c_size_t,
                                  c_void_p]),
    "qmc_reduce_partials": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_size_t, c_void_p, c_void_p,
                                    c_void_p]),
    "qmc_probe_precision": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_int64, c_void_p,
                                    c_void_p]),
    "qmc_probe_islands": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_int64, c_void_p,
                                  c_void_p, c_void_p]),
    "qmc_choose_precision": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_double,
                                     c_double, c_void_p, c_void_p]),
    "qmc_eval_sums_noalloc": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
    "qmc_autotune_scratch_bytes": (c_size_t, [c_void_p, POINTER(qmc_pass)]),
    "qmc_autotune": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_void_p, c_size_t,
                             POINTER(qmc_tune_result), c_void_p]),
    "qmc_autotune_clear": (c_int, []),
    "qmc_gen_source": (c_int, [c_void_p, c_int32, c_void_p, c_size_t, POINTER(c_size_t)]),
    "qmc_gen_compile": (c_int, [c_void_p, c_int32, c_int32, POINTER(qmc_gen_info)]),
    "qmc_eval_points": (c_int, [c_void_p, c_void_p, c_int32, POINTER(qmc_pass), c_void_p, c_double, c_void_p,
                                c_int64, c_void_p, c_void_p, c_void_p]),
    "qmc_builtin_lattices": (c_int, [POINTER(qmc_lattice), c_int32]),
    "qmc_combine": (c_int, [c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_void_p, c_void_p]),
    "qmc_combine_sectors": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "qmc_create": (c_int, [POINTER(c_void_p), c_int32, c_size_t, c_void_p]),
    "qmc_destroy": (c_int, [c_void_p]),
    "qmc_load_sectors": (c_int, [c_void_p, c_void_p, c_size_t, POINTER(c_int32)]),
    "qmc_set_kinematics": (c_int, [c_void_p, c_int32, POINTER(c_double), c_int32, c_int32, c_int32]),
    "qmc_eval_sums_host": (c_int, [c_void_p, c_void_p, POINTER(qmc_pass), c_void_p, c_void_p, c_void_p, c_void_p]),
    "qmc_submit": (c_int, [c_void_p, c_int32, POINTER(c_double), c_int32, c_int32, c_int32, POINTER(qmc_options),
                           POINTER(c_int64)]),
    "qmc_poll": (c_int, [c_void_p, c_int64, POINTER(qmc_result)]),
    "qmc_cancel": (c_int, [c_void_p, c_int64]),
    "qmc_serving_stats_get": (c_int, [c_void_p, POINTER(qmc_serving_stats)]),
    "qmc_integrate": (c_int, [c_void_p, c_int32, POINTER(qmc_options), POINTER(qmc_result)]),
}

_lib = None


class QMCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


def lib():
    """The loaded library; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"qmcfi CUDA library not built ({LIB}); run `python -m paper_1508_02512_gb300.build`")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().qmc_strerror(status).decode()


def check(status: int, where: str) -> int:
    if status < 0:
        raise QMCError(status, where)
    return status
