"""ctypes wrapper of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY.  Built with gcc (``build()``), loaded lazily.  Every
function takes plain numpy arrays; none of them touches the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB


def build_command(openmp: bool = True) -> list[str]:
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _LIB, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    return cmd


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_liboracle.so`` next to it (gcc, FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.run(build_command(), check=True)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.oracle_cost_at.restype = ctypes.c_uint32
            lib.oracle_cost_at.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P, P]
            lib.oracle_cost_samples.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int64, P, P]
            lib.oracle_cost_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
            lib.oracle_evolve.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int, P]
            lib.oracle_success_prob.argtypes = [ctypes.c_int, P, P, P, P]
            lib.oracle_grad.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P]
            lib.oracle_sample.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P]
            lib.oracle_running_time.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _clauses(var, neg):
    var = np.ascontiguousarray(var, dtype=np.int32)
    neg = np.ascontiguousarray(neg, dtype=np.uint8)
    if var.ndim != 2 or var.shape != neg.shape:
        raise ValueError("var and neg must both be [m, k]")
    return var, neg


def cost_table(n: int, var, neg):
    """Returns (C as uint16 [2^n], number of solutions, max C)."""
    var, neg = _clauses(var, neg)
    m, k = var.shape
    cost = np.empty(1 << n, dtype=np.uint16)
    n_sol = ctypes.c_uint64()
    mx = ctypes.c_uint32()
    rc = _load().oracle_cost_table(n, m, max(k, 1), _ptr(var), _ptr(neg), _ptr(cost),
                                   ctypes.byref(n_sol), ctypes.byref(mx))
    if rc != 0:
        raise ValueError(f"oracle_cost_table failed ({rc})")
    return cost, int(n_sol.value), int(mx.value)


def cost_samples(var, neg, xs) -> np.ndarray:
    """C(x) for each x in ``xs`` (uint64), evaluated one by one."""
    var, neg = _clauses(var, neg)
    m, k = var.shape
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    out = np.empty(xs.shape[0], dtype=np.uint32)
    rc = _load().oracle_cost_samples(m, max(k, 1), _ptr(var), _ptr(neg), xs.shape[0], _ptr(xs), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_cost_samples failed ({rc})")
    return out


def count_solutions(inst) -> int:
    """Number of x with C(x) = 0 (brute force over 2^n); ``inst`` has n, var, neg."""
    _, sol, _ = cost_table(inst.n, inst.var, inst.neg)
    return sol


def _angles(gamma, beta):
    gamma = np.ascontiguousarray(gamma, dtype=np.float64).reshape(-1)
    beta = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1)
    if gamma.shape != beta.shape:
        raise ValueError("gamma and beta must have the same length")
    return gamma, beta


def evolve(n: int, cost, gamma, beta, sign: int = 1) -> np.ndarray:
    """The output state prod_i U_B(beta_i) U_C(gamma_i) |+>^n as complex128 [2^n]."""
    cost = np.ascontiguousarray(cost, dtype=np.uint16)
    gamma, beta = _angles(gamma, beta)
    psi = np.empty(1 << n, dtype=np.complex128)
    rc = _load().oracle_evolve(n, _ptr(cost), gamma.shape[0], _ptr(gamma), _ptr(beta), sign, _ptr(psi))
    if rc != 0:
        raise ValueError(f"oracle_evolve failed ({rc})")
    return psi


def success_prob(n: int, cost, psi):
    """(p_succ, norm) of a complex128 state."""
    cost = np.ascontiguousarray(cost, dtype=np.uint16)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    ps = ctypes.c_double()
    nm = ctypes.c_double()
    rc = _load().oracle_success_prob(n, _ptr(cost), _ptr(psi), ctypes.byref(ps), ctypes.byref(nm))
    if rc != 0:
        raise ValueError(f"oracle_success_prob failed ({rc})")
    return ps.value, nm.value


def grad(n: int, cost, gamma, beta, sign: int = 1):
    """(p_succ, dp/dgamma [p], dp/dbeta [p]) by stored-state reverse mode."""
    cost = np.ascontiguousarray(cost, dtype=np.uint16)
    gamma, beta = _angles(gamma, beta)
    p = gamma.shape[0]
    dg = np.zeros(p)
    db = np.zeros(p)
    ps = ctypes.c_double()
    rc = _load().oracle_grad(n, _ptr(cost), p, _ptr(gamma), _ptr(beta), sign, ctypes.byref(ps), _ptr(dg), _ptr(db))
    if rc != 0:
        raise ValueError(f"oracle_grad failed ({rc})")
    return ps.value, dg, db


def sample(n: int, psi, u) -> np.ndarray:
    """Draws x_j = min{x : F(x) > u_j F_total} from |psi|^2 (inverse CDF in index order); uint64 [k]."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    xs = np.empty(u.shape[0], dtype=np.uint64)
    rc = _load().oracle_sample(n, _ptr(psi), u.shape[0], _ptr(u), _ptr(xs))
    if rc != 0:
        raise ValueError(f"oracle_sample failed ({rc})")
    return xs


def running_time(n: int, cost, psi, u) -> int:
    """1 + index of the first draw that satisfies the instance (C = 0), 0 if none does."""
    cost = np.ascontiguousarray(cost, dtype=np.uint16)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    rt = ctypes.c_int64()
    rc = _load().oracle_running_time(n, _ptr(cost), _ptr(psi), u.shape[0], _ptr(u), ctypes.byref(rt))
    if rc != 0:
        raise ValueError(f"oracle_running_time failed ({rc})")
    return rt.value
