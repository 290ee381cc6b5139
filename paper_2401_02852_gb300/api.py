"""Python binding of the C ABI (``include/qaoa.h``): argument marshalling only.

Device memory comes from torch; every step of the path runs in the library's
CUDA kernels.  Tensors must be contiguous CUDA tensors on the current device.
Streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import C64, C128, MIXER_PAPER, MIXER_RX2B, Z2_HALF, NaesatInstance, check, load

DTYPES = {"c64": C64, "c128": C128, C64: C64, C128: C128, torch.complex64: C64, torch.complex128: C128}
TORCH_DTYPE = {C64: torch.complex64, C128: torch.complex128}


def dtype_code(dtype) -> int:
    try:
        return DTYPES[dtype]
    except KeyError:
        raise ValueError(f"dtype must be 'c64' or 'c128', got {dtype!r}") from None


def _stream(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def _np_ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


class _Inst:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, inst):
        self.var = np.ascontiguousarray(inst.var, dtype=np.int32)
        self.neg = np.ascontiguousarray(inst.neg, dtype=np.uint8)
        m = int(self.var.shape[0])
        k = int(self.var.shape[1]) if self.var.ndim == 2 else int(inst.k)
        self.s = NaesatInstance(int(inst.n), m, k, _np_ptr(self.var).value or 0, _np_ptr(self.neg).value or 0)


def cost_table(inst, out: Optional[torch.Tensor] = None, stream=None, stats: bool = True):
    """C(x) for all x as a CUDA uint8 tensor [2^n]; returns (cost, n_sol, max_cost).

    With ``stats=False`` the call does not wait for the device (n_sol and
    max_cost are then None, unless m > 255 where the range check needs them).
    """
    n = int(inst.n)
    if out is None:
        out = torch.empty(1 << n, dtype=torch.uint8, device="cuda")
    ci = _Inst(inst)
    ns = ctypes.c_uint64()
    mx = ctypes.c_uint32()
    args = (ctypes.byref(ns), ctypes.byref(mx)) if stats else (None, None)
    check(load().naesat_cost_table(ctypes.byref(ci.s), _ptr(out), *args, _stream(stream)))
    return out, (int(ns.value) if stats else None), (int(mx.value) if stats else None)


def cost_table_half(inst, out: Optional[torch.Tensor] = None, stream=None, stats: bool = True):
    """C(x) for x < 2^(n-1) (the halved-state table); n_sol / max_cost of the full table."""
    n = int(inst.n)
    if out is None:
        out = torch.empty(1 << (n - 1), dtype=torch.uint8, device="cuda")
    ci = _Inst(inst)
    ns = ctypes.c_uint64()
    mx = ctypes.c_uint32()
    args = (ctypes.byref(ns), ctypes.byref(mx)) if stats else (None, None)
    check(load().naesat_cost_table_half(ctypes.byref(ci.s), _ptr(out), *args, _stream(stream)))
    return out, (int(ns.value) if stats else None), (int(mx.value) if stats else None)


def cost_table_batch(insts: Sequence, out: Optional[torch.Tensor] = None, stream=None):
    """Cost tables of several instances of one n: uint8 [B, 2^n], n_sol [B], max [B]."""
    B = len(insts)
    n = int(insts[0].n)
    if out is None:
        out = torch.empty((B, 1 << n), dtype=torch.uint8, device="cuda")
    cis = [_Inst(i) for i in insts]
    arr = (NaesatInstance * B)(*[c.s for c in cis])
    ns = np.zeros(B, dtype=np.uint64)
    mx = np.zeros(B, dtype=np.uint32)
    check(load().naesat_cost_table_batch(B, ctypes.byref(arr), _ptr(out), _np_ptr(ns), _np_ptr(mx), _stream(stream)))
    return out, ns, mx


def evolve(n: int, cost: torch.Tensor, m: int, gamma, beta, dtype="c64", flags: int = MIXER_PAPER,
           out: Optional[torch.Tensor] = None, want: bool = True, stream=None):
    """prod_l U_B(beta_l) U_C(gamma_l) |+>^n; returns (state, p_succ, norm).

    ``want=False`` skips the fused reduction and does not wait for the device.
    With ``flags & Z2_HALF`` the state holds the 2^(n-1) amplitudes with bit
    n-1 clear and ``cost`` is the half table (``cost_table_half``).
    """
    code = dtype_code(dtype)
    g, b = _f64(gamma), _f64(beta)
    if g.shape != b.shape:
        raise ValueError("gamma and beta differ in length")
    if out is None:
        out = torch.empty(1 << (n - 1 if flags & Z2_HALF else n), dtype=TORCH_DTYPE[code], device="cuda")
    ps, nm = ctypes.c_double(), ctypes.c_double()
    res = (ctypes.byref(ps), ctypes.byref(nm)) if want else (None, None)
    check(load().qaoa_evolve(n, _ptr(cost), int(m), g.shape[0], _np_ptr(g), _np_ptr(b), code, flags, _ptr(out),
                             *res, _stream(stream)))
    return out, (ps.value if want else None), (nm.value if want else None)


def evolve_batch(n: int, costs: torch.Tensor, m_max: int, gamma, beta, dtype="c64", flags: int = MIXER_PAPER,
                 out: Optional[torch.Tensor] = None, stream=None):
    """Batched evolution with shared angles: states [B, 2^n], p_succ [B], norm [B]."""
    code = dtype_code(dtype)
    B = int(costs.shape[0])
    g, b = _f64(gamma), _f64(beta)
    if out is None:
        out = torch.empty((B, 1 << (n - 1 if flags & Z2_HALF else n)), dtype=TORCH_DTYPE[code], device="cuda")
    ps = np.zeros(B)
    nm = np.zeros(B)
    check(load().qaoa_evolve_batch(B, n, _ptr(costs), int(m_max), g.shape[0], _np_ptr(g), _np_ptr(b), code, flags,
                                   _ptr(out), _np_ptr(ps), _np_ptr(nm), _stream(stream)))
    return out, ps, nm


def success_prob(n: int, cost: torch.Tensor, state: torch.Tensor, stream=None):
    """(p_succ, norm) of a device state, FP64 reduction."""
    code = dtype_code(state.dtype)
    ps, nm = ctypes.c_double(), ctypes.c_double()
    check(load().qaoa_success_prob(n, _ptr(cost), _ptr(state), code, ctypes.byref(ps), ctypes.byref(nm),
                                   _stream(stream)))
    return ps.value, nm.value


def _uniforms(u, count: int) -> torch.Tensor:
    u = torch.as_tensor(u, dtype=torch.float64)
    u = u.to("cuda").contiguous()
    if u.numel() != count:
        raise ValueError(f"expected {count} uniforms, got {u.numel()}")
    return u


def sample(n: int, state: torch.Tensor, u, flags: int = 0, out: Optional[torch.Tensor] = None, stream=None):
    """Bitstrings drawn from |state|^2 by inverse CDF, one per uniform in `u`
    (Sec. "Running Times"); int64 device tensor [k] (x < 2^n)."""
    k = int(np.prod(np.shape(u)))
    du = _uniforms(u, k)
    if out is None:
        out = torch.empty(k, dtype=torch.int64, device="cuda")
    check(load().qaoa_sample(n, _ptr(state), dtype_code(state.dtype), flags, k, _ptr(du), _ptr(out),
                             _stream(stream)))
    return out


def running_time(n: int, cost: torch.Tensor, state: torch.Tensor, u, flags: int = 0, stream=None) -> int:
    """1 + index of the first draw (one per uniform) that satisfies the
    instance, or 0 when none does."""
    k = int(np.prod(np.shape(u)))
    du = _uniforms(u, k)
    rt = ctypes.c_int64()
    check(load().qaoa_running_time(n, _ptr(cost), _ptr(state), dtype_code(state.dtype), flags, k, _ptr(du),
                                   ctypes.byref(rt), None, _stream(stream)))
    return rt.value


def running_time_batch(n: int, costs: torch.Tensor, states: torch.Tensor, u, flags: int = 0, stream=None):
    """Running times of a batch (same n): u has shape [batch, k]; int64 numpy [batch]."""
    batch = states.shape[0]
    k = int(np.prod(np.shape(u))) // batch
    du = _uniforms(u, batch * k)
    rt = np.zeros(batch, dtype=np.int64)
    check(load().qaoa_running_time_batch(batch, n, _ptr(costs), _ptr(states), dtype_code(states.dtype), flags, k,
                                         _ptr(du), _np_ptr(rt), _stream(stream)))
    return rt


def grad(n: int, cost: torch.Tensor, m: int, gamma, beta, dtype="c64", flags: int = MIXER_PAPER,
         work: Optional[tuple] = None, stream=None):
    """(p_succ, dp/dgamma [p], dp/dbeta [p]) by the recompute-backward adjoint sweep."""
    code = dtype_code(dtype)
    g, b = _f64(gamma), _f64(beta)
    p = g.shape[0]
    if work is None:
        work = (torch.empty(1 << n, dtype=TORCH_DTYPE[code], device="cuda"),
                torch.empty(1 << n, dtype=TORCH_DTYPE[code], device="cuda"))
    ps = ctypes.c_double()
    dg = np.zeros(p)
    db = np.zeros(p)
    check(load().qaoa_grad(n, _ptr(cost), int(m), p, _np_ptr(g), _np_ptr(b), code, flags, _ptr(work[0]),
                           _ptr(work[1]), ctypes.byref(ps), _np_ptr(dg), _np_ptr(db), _stream(stream)))
    return ps.value, dg, db


def grad_batch(n: int, costs: torch.Tensor, m_max: int, gamma, beta, dtype="c64", flags: int = MIXER_PAPER,
               work: Optional[tuple] = None, stream=None):
    """Batched gradients with shared angles: p_succ [B], dgamma [B, p], dbeta [B, p]."""
    code = dtype_code(dtype)
    B = int(costs.shape[0])
    g, b = _f64(gamma), _f64(beta)
    p = g.shape[0]
    if work is None:
        work = (torch.empty((B, 1 << n), dtype=TORCH_DTYPE[code], device="cuda"),
                torch.empty((B, 1 << n), dtype=TORCH_DTYPE[code], device="cuda"))
    ps = np.zeros(B)
    dg = np.zeros((B, p))
    db = np.zeros((B, p))
    check(load().qaoa_grad_batch(B, n, _ptr(costs), int(m_max), p, _np_ptr(g), _np_ptr(b), code, flags,
                                 _ptr(work[0]), _ptr(work[1]), _np_ptr(ps), _np_ptr(dg), _np_ptr(db),
                                 _stream(stream)))
    return ps, dg, db


def psucc_host(inst, gamma, beta, dtype="c64", flags: int = MIXER_PAPER, work: Optional[dict] = None, stream=None):
    """End to end from host memory: clauses in, (p_succ, norm, n_sol) out.

    Runs the cost table, the evolution and the fused reduction through the C ABI;
    ``work`` may hold reusable device buffers ('cost', 'state').
    """
    n = int(inst.n)
    work = {} if work is None else work
    code = dtype_code(dtype)
    half = bool(flags & Z2_HALF)  # the halved table and state (global-flip symmetry)
    size = 1 << (n - 1 if half else n)
    if "cost" not in work or work["cost"].numel() != size:
        work["cost"] = torch.empty(size, dtype=torch.uint8, device="cuda")
    if "state" not in work or work["state"].numel() != size or work["state"].dtype != TORCH_DTYPE[code]:
        work["state"] = torch.empty(size, dtype=TORCH_DTYPE[code], device="cuda")
    table = cost_table_half if half else cost_table
    cost, _, _ = table(inst, out=work["cost"], stream=stream, stats=False)
    _, ps, nm = evolve(n, cost, inst.var.shape[0], gamma, beta, dtype, flags, out=work["state"], stream=stream)
    return ps, nm


def plan(n: int, dtype="c64", flags: int = 0):
    """Pass plan: list of (group_lo, group_bits, row_bits) per HBM pass of one layer."""
    lo = (ctypes.c_int * 8)()
    bits = (ctypes.c_int * 8)()
    row = (ctypes.c_int * 8)()
    k = check(load().qaoa_plan(n, dtype_code(dtype), flags, lo, bits, row))
    return [(lo[i], bits[i], row[i]) for i in range(k)]


def pass_schedule(n: int, p: int, dtype="c64", flags: int = 0):
    """Launch sequence of an evolution: list of (pass index, layer, mode)."""
    cap = max(1, p * 8 + 1)
    idx = (ctypes.c_int * cap)()
    lay = (ctypes.c_int * cap)()
    mod = (ctypes.c_int * cap)()
    k = check(load().qaoa_pass_schedule(n, p, dtype_code(dtype), flags, cap, idx, lay, mod))
    return [(idx[i], lay[i], mod[i]) for i in range(k)]


class Profiler:
    """Per-kernel CUDA-event timing of every library launch inside the block."""

    KINDS = 16

    def __enter__(self):
        load().qaoa_profile_read(0, None, None)
        load().qaoa_profile_enable(1)
        return self

    def __exit__(self, *exc):
        lib = load()
        lib.qaoa_profile_enable(0)
        launches = (ctypes.c_uint64 * self.KINDS)()
        ms = (ctypes.c_double * self.KINDS)()
        k = check(lib.qaoa_profile_read(self.KINDS, launches, ms))
        self.stats = {lib.qaoa_kernel_name(i).decode(): (int(launches[i]), float(ms[i])) for i in range(k)
                      if launches[i]}
        return False


def launch_count() -> int:
    return int(load().qaoa_launch_count())
