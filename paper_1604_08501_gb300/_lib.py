"""ctypes declarations of the C ABI in ``include/numa_vol.h``.

The library is the in-tree ``libnumavol.so`` built by ``build.py``.  There is
no fallback: if the library is missing or does not load, every entry point
raises."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

NUMA_OK, NUMA_EINVAL, NUMA_ENOMEM, NUMA_ECUDA, NUMA_EUNSUPPORTED, NUMA_ETIMEOUT, NUMA_ELIMIT = 0, -1, -2, -3, -4, -5, -6
NUMA_NOALLOC_MAX_INSTANCES = 64
NUMA_MAX_N = 7
NUMA_MAX_N_FP64 = 15
NUMA_FP64, NUMA_MIXED, NUMA_DF64 = 0, 1, 2
NUMA_SWEEP_CUDA_CORES, NUMA_SWEEP_TENSOR_TF32, NUMA_SWEEP_AUTO = 0, 1, 2

_ERRNAMES = {NUMA_EINVAL: "NUMA_EINVAL", NUMA_ENOMEM: "NUMA_ENOMEM",
             NUMA_ECUDA: "NUMA_ECUDA", NUMA_EUNSUPPORTED: "NUMA_EUNSUPPORTED",
             NUMA_ETIMEOUT: "NUMA_ETIMEOUT", NUMA_ELIMIT: "NUMA_ELIMIT"}

_DP = C.POINTER(C.c_double)


class numa_constants(C.Structure):
    _fields_ = [("p0", C.c_double), ("R", C.c_double), ("cp", C.c_double), ("grav", C.c_double)]


class numa_mesh(C.Structure):
    _fields_ = [("num_elements", C.c_int64), ("N", C.c_int), ("num_tracers", C.c_int)]


class numa_geometry(C.Structure):
    _fields_ = [("g", C.c_void_p * 9), ("Jinv", C.c_void_p), ("rho_ref", C.c_void_p),
                ("rhotheta_ref", C.c_void_p)]


class numa_request_info(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double)]


class numa_engine_counters(C.Structure):
    _fields_ = [("queued", C.c_int), ("resident", C.c_int), ("bytes_used", C.c_size_t),
                ("bytes_budget", C.c_size_t), ("completed", C.c_int64), ("rounds", C.c_int64),
                ("point_stages", C.c_double)]


class numa_batch_config(C.Structure):
    _fields_ = [("tile", C.c_int * 9), ("sweep", C.c_int * 9), ("ctas_per_sm", C.c_int),
                ("costliest_first", C.c_int), ("state_in_tmem", C.c_int),
                ("tuned_ms_per_step", C.c_double),
                ("tuned_candidates", C.c_int)]


NUMA_REQ_QUEUED, NUMA_REQ_RUNNING, NUMA_REQ_DONE, NUMA_REQ_CANCELLED = 0, 1, 2, 3


class NumaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load() -> C.CDLL:
    """Load ``libnumavol.so``; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(
            f"{LIB} is not built: call __graft_entry__.build() (or "
            "paper_1604_08501_gb300.build.build()) first; there is no CPU fallback")
    lib = C.CDLL(LIB)
    lib.numa_vol_create.argtypes = [C.POINTER(numa_mesh), C.POINTER(numa_geometry),
                                    C.POINTER(numa_constants), C.c_int, C.POINTER(C.c_void_p)]
    lib.numa_vol_create.restype = C.c_int
    lib.numa_vol_rhs.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.numa_vol_rhs.restype = C.c_int
    lib.numa_vol_rhs_host.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.numa_vol_rhs_host.restype = C.c_int
    lib.numa_vol_status.argtypes = [C.c_void_p, C.c_void_p]
    lib.numa_vol_status.restype = C.c_int
    lib.numa_vol_destroy.argtypes = [C.c_void_p]
    lib.numa_vol_destroy.restype = None
    lib.numa_vol_last_error.argtypes = []
    lib.numa_vol_last_error.restype = C.c_char_p
    lib.numa_vol_kernel_name.argtypes = [C.c_void_p]
    lib.numa_vol_set_sweep.argtypes = [C.c_void_p, C.c_int]
    lib.numa_vol_set_sweep.restype = C.c_int
    lib.numa_vol_kernel_name.restype = C.c_char_p
    lib.numa_vol_diff_matrix.argtypes = [C.c_int, _DP]
    lib.numa_vol_diff_matrix.restype = C.c_int
    lib.numa_batch_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    lib.numa_batch_add.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
    lib.numa_batch_clear.argtypes = [C.c_void_p]
    lib.numa_batch_size.argtypes = [C.c_void_p]
    lib.numa_batch_advance.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p]
    lib.numa_batch_autotune.argtypes = [C.c_void_p, C.c_void_p]
    lib.numa_batch_tile.argtypes = [C.c_void_p, C.c_int]
    lib.numa_batch_set_sweep.argtypes = [C.c_void_p, C.c_int]
    lib.numa_batch_sweep.argtypes = [C.c_void_p]
    lib.numa_batch_sweep_of.argtypes = [C.c_void_p, C.c_int]
    lib.numa_batch_status.argtypes = [C.c_void_p, C.c_void_p]
    lib.numa_batch_get_config.argtypes = [C.c_void_p, C.POINTER(numa_batch_config)]
    lib.numa_batch_set_config.argtypes = [C.c_void_p, C.POINTER(numa_batch_config)]
    lib.numa_batch_last_error.restype = C.c_char_p
    lib.numa_batch_destroy.argtypes = [C.c_void_p]
    lib.numa_batch_destroy.restype = None
    lib.numa_vol_selftest_wait.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p]
    lib.numa_vol_selftest_wait.restype = C.c_int
    lib.numa_engine_create.argtypes = [C.c_int, C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]
    lib.numa_engine_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_double, C.POINTER(C.c_int64)]
    lib.numa_engine_cancel.argtypes = [C.c_void_p, C.c_int64]
    lib.numa_engine_progress.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_int,
                                         C.POINTER(C.c_int)]
    lib.numa_engine_drain.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_int,
                                      C.POINTER(C.c_int)]
    lib.numa_engine_query.argtypes = [C.c_void_p, C.c_int64, C.POINTER(numa_request_info)]
    lib.numa_engine_checkpoint.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_int)]
    lib.numa_engine_set_round_steps.argtypes = [C.c_void_p, C.c_int]
    lib.numa_engine_set_round_policy.argtypes = [C.c_void_p, C.c_int]
    lib.numa_engine_stats.argtypes = [C.c_void_p, C.POINTER(numa_engine_counters)]
    lib.numa_engine_last_error.restype = C.c_char_p
    lib.numa_engine_destroy.argtypes = [C.c_void_p]
    lib.numa_engine_destroy.restype = None
    for name in ("numa_engine_create", "numa_engine_submit", "numa_engine_cancel",
                 "numa_engine_progress", "numa_engine_drain", "numa_engine_query",
                 "numa_engine_stats",
                 "numa_engine_checkpoint", "numa_engine_set_round_steps",
                 "numa_engine_set_round_policy"):
        getattr(lib, name).restype = C.c_int
    lib.numa_batch_advance_noalloc.argtypes = [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                               C.c_int, C.c_double, C.c_void_p]
    lib.numa_batch_advance_noalloc.restype = C.c_int
    for name in ("numa_batch_create", "numa_batch_add", "numa_batch_clear", "numa_batch_size",
                 "numa_batch_advance", "numa_batch_autotune", "numa_batch_tile",
                 "numa_batch_set_sweep", "numa_batch_sweep", "numa_batch_sweep_of",
                 "numa_batch_status", "numa_batch_get_config", "numa_batch_set_config"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(code: int) -> None:
    if code != NUMA_OK:
        msg = load().numa_vol_last_error().decode(errors="replace")
        raise NumaError(code, msg)


def check_engine(code: int) -> None:
    if code != NUMA_OK:
        msg = load().numa_engine_last_error().decode(errors="replace")
        raise NumaError(code, msg)


def check_batch(code: int) -> None:
    if code != NUMA_OK:
        msg = load().numa_batch_last_error().decode(errors="replace")
        raise NumaError(code, msg)
