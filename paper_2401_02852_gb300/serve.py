"""Python binding of the serving loop (``qaoa_server_*`` in include/qaoa.h).

The scheduler, admission, packing and streams are native (csrc/serve.cu);
this module marshals arguments and adds a replay driver that submits a
request stream at its arrival times and collects latency statistics.
"""
from __future__ import annotations

import ctypes
import threading
import time
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import QAOA_OK, QAOA_PENDING, Result, ServerOpts, check, load
from .api import _Inst, dtype_code


@dataclass
class ServeResult:
    ticket: int
    p_succ: float
    norm: float
    n_sol: int
    max_cost: int
    status: int
    t_submit_ns: int
    t_start_ns: int
    t_done_ns: int

    @property
    def latency_s(self) -> float:
        return (self.t_done_ns - self.t_submit_ns) * 1e-9


def _result(ticket: int, r: Result) -> ServeResult:
    return ServeResult(ticket, r.p_succ, r.norm, int(r.n_sol), int(r.max_cost), int(r.status), int(r.t_submit_ns),
                       int(r.t_start_ns), int(r.t_done_ns))


class Server:
    """A native serving loop on one device (continuous batching)."""

    def __init__(self, dtype="c64", hbm_budget_bytes: int = 0, max_batch: int = 256, n_streams: int = 4,
                 small_n_max: int = 0, flags: int = 0, device: int = 0, max_n: int = 30):
        opts = ServerOpts(hbm_budget_bytes, max_batch, n_streams, dtype_code(dtype), small_n_max, flags, device,
                          max_n)
        self._h = ctypes.c_void_p()
        check(load().qaoa_server_create(ctypes.byref(opts), ctypes.byref(self._h)))

    def submit(self, inst, gamma, beta) -> int:
        ci = _Inst(inst)
        g = np.ascontiguousarray(gamma, dtype=np.float64)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        t = ctypes.c_uint64()
        check(load().qaoa_serve_submit(self._h, ctypes.byref(ci.s), int(g.shape[0]), g.ctypes.data, b.ctypes.data,
                                       ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int) -> Optional[ServeResult]:
        r = Result()
        rc = check(load().qaoa_serve_poll(self._h, ticket, ctypes.byref(r)))
        return None if rc == QAOA_PENDING else _result(ticket, r)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> ServeResult:
        r = Result()
        check(load().qaoa_serve_wait(self._h, ticket, ctypes.byref(r), float(timeout_s)))
        return _result(ticket, r)

    def cancel(self, ticket: int) -> bool:
        return check(load().qaoa_serve_cancel(self._h, ticket)) == QAOA_OK

    def stats(self) -> dict:
        c = (ctypes.c_uint64 * 8)()
        check(load().qaoa_server_stats(self._h, c))
        keys = ["submitted", "completed", "packed_launches", "single_launches", "peak_bytes", "cancelled", "errors",
                "grouped_requests"]
        return dict(zip(keys, (int(v) for v in c)))

    def issue_time(self) -> dict:
        """Host time spent issuing work and its share of the time since the first admission."""
        ns, k, span = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(load().qaoa_server_issue_time(self._h, ctypes.byref(ns), ctypes.byref(k), ctypes.byref(span)))
        return {"issue_s": ns.value * 1e-9, "issues": int(k.value), "span_s": span.value * 1e-9,
                "issue_share": ns.value / span.value if span.value else None,
                "mean_issue_us": ns.value / k.value / 1e3 if k.value else None}

    def close(self):
        if self._h:
            check(load().qaoa_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def replay(server: Server, requests: Sequence, time_scale: float = 1.0, timeout_s: float = 600.0):
    """Submits each request at its arrival time (scaled) and waits for all.

    Returns (results by request index, wall seconds from the first arrival to
    the last completion)."""
    tickets = [None] * len(requests)
    t0 = time.perf_counter()
    for i, rq in enumerate(requests):
        due = t0 + rq.arrival_s * time_scale
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        tickets[i] = server.submit(rq.instance, rq.gamma, rq.beta)
    out = [server.wait(t, timeout_s) for t in tickets]
    wall = (max(r.t_done_ns for r in out) - min(r.t_submit_ns for r in out)) * 1e-9
    return out, wall


def one_per_launch(requests: Sequence, dtype="c64", time_scale: float = 1.0, flags: int = 0, half_above: int = 14):
    """Baseline on the same GPU: one request at a time, each its own cost-table
    and evolution launches, in arrival order (queueing delay included).  With
    QAOA_Z2_HALF in ``flags`` the requests with n > ``half_above`` run on the
    halved state, as a server with that flag runs its unpacked requests."""
    import torch

    from . import api

    lat = []
    results = []
    t0 = time.perf_counter()
    work = {}
    for rq in requests:
        due = t0 + rq.arrival_s * time_scale
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        arrival = max(due, t0)
        f = flags if rq.instance.n > half_above else flags & ~_lib.Z2_HALF
        ps, nm = api.psucc_host(rq.instance, rq.gamma, rq.beta, dtype, flags=f, work=work)
        torch.cuda.synchronize()
        done = time.perf_counter()
        lat.append(done - arrival)
        results.append(ps)
    wall = time.perf_counter() - t0 - requests[0].arrival_s * time_scale
    return results, np.array(lat), wall


def latency_summary(lat_s: np.ndarray, wall_s: float, count: int) -> dict:
    return {"inst_per_s": count / wall_s, "p50_ms": float(np.percentile(lat_s, 50) * 1e3),
            "p99_ms": float(np.percentile(lat_s, 99) * 1e3), "mean_ms": float(lat_s.mean() * 1e3),
            "count": count, "wall_s": wall_s}
