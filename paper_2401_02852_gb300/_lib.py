"""ctypes loader of ``libqaoa.so``: argument marshalling only.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2401_02852_gb300._build``).  There is no fallback: when the
library is missing or cannot be loaded every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqaoa.so")

QAOA_OK = 0
QAOA_PENDING = 1
ERRORS = {-1: "EINVAL", -2: "ERANGE", -3: "ENOMEM", -4: "ECUDA", -5: "ETIMEOUT", -6: "ECANCELLED", -7: "ENOTFOUND"}
C64, C128 = 0, 1
MIXER_PAPER, MIXER_RX2B = 0, 1
Z2_HALF = 2
DF64 = 4


class QaoaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class NaesatInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("k", ctypes.c_int32),
                ("var", ctypes.c_void_p), ("neg", ctypes.c_void_p)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("n_streams", ctypes.c_int),
                ("dtype", ctypes.c_int), ("small_n_max", ctypes.c_int), ("flags", ctypes.c_int),
                ("device", ctypes.c_int), ("max_n", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("p_succ", ctypes.c_double), ("norm", ctypes.c_double), ("n_sol", ctypes.c_uint64),
                ("max_cost", ctypes.c_uint32), ("status", ctypes.c_int32), ("t_submit_ns", ctypes.c_uint64),
                ("t_start_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]


P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
# name -> (restype, argtypes); mirrors include/qaoa.h
SIGNATURES = {
    "qaoa_last_error": (ctypes.c_char_p, []),
    "qaoa_version": (I, []),
    "qaoa_release_scratch": (I, []),
    "naesat_cost_table": (I, [P, P, P, P, P]),
    "naesat_cost_table_half": (I, [P, P, P, P, P]),
    "naesat_cost_table_batch": (I, [I, P, P, P, P, P]),
    "qaoa_evolve": (I, [I, P, I, I, P, P, I, I, P, P, P, P]),
    "qaoa_evolve_batch": (I, [I, I, P, I, I, P, P, I, I, P, P, P, P]),
    "qaoa_success_prob": (I, [I, P, P, I, P, P, P]),
    "qaoa_success_prob_noalloc": (I, [I, P, P, I, P, P, P]),
    "qaoa_sample": (I, [I, P, I, I, I, P, P, P]),
    "qaoa_running_time": (I, [I, P, P, I, I, I, P, P, P, P]),
    "qaoa_running_time_batch": (I, [I, I, P, P, I, I, I, P, P, P]),
    "qaoa_grad": (I, [I, P, I, I, P, P, I, I, P, P, P, P, P, P]),
    "qaoa_grad_batch": (I, [I, I, P, I, I, P, P, I, I, P, P, P, P, P, P]),
    "qaoa_server_create": (I, [P, P]),
    "qaoa_serve_submit": (I, [P, P, I, P, P, P]),
    "qaoa_serve_poll": (I, [P, ctypes.c_uint64, P]),
    "qaoa_serve_wait": (I, [P, ctypes.c_uint64, P, D]),
    "qaoa_serve_cancel": (I, [P, ctypes.c_uint64]),
    "qaoa_server_stats": (I, [P, P]),
    "qaoa_server_issue_time": (I, [P, P, P, P]),
    "qaoa_server_destroy": (I, [P]),
    "qaoa_plan": (I, [I, I, I, P, P, P]),
    "qaoa_pass_schedule": (I, [I, I, I, I, I, P, P, P]),
    "qaoa_adjoint_schedule": (I, [I, I, I, I, P, P, P]),
    "qaoa_profile_enable": (I, [I]),
    "qaoa_profile_read": (I, [I, P, P]),
    "qaoa_kernel_name": (ctypes.c_char_p, [I]),
    "qaoa_launch_count": (ctypes.c_uint64, []),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Loads the built library (raises if it is missing: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int) -> int:
    if rc < 0:
        raise QaoaError(rc, load().qaoa_last_error().decode())
    return rc
