"""Angle training with the adjoint gradient (Sec. "QAOA Procedure": fixed angles
are trained with Adam on an objective of the success probability).

``QaoaPsucc`` is a ``torch.autograd.Function`` over the shared angles of a batch
of instances: its forward runs the library's batched adjoint sweep, which
returns p_succ and d p_succ / d(gamma, beta) together; its backward contracts
the stored per-instance gradients with the incoming gradient.  Angles live on
the host as float64 tensors (2p numbers); states stay on the device.
"""
from __future__ import annotations

import json
import os
from typing import Optional

import numpy as np
import torch

from . import api


class QaoaPsucc(torch.autograd.Function):
    """p_succ [B] of B instances (cost tables [B, 2^n]) as a function of the
    shared angles gamma [p], beta [p] (float64, CPU)."""

    @staticmethod
    def forward(ctx, gamma, beta, costs, n, m, dtype, flags, work):
        ps, dg, db = api.grad_batch(n, costs, m, gamma.detach().numpy(), beta.detach().numpy(), dtype, flags,
                                    work=work)
        ctx.save_for_backward(torch.from_numpy(dg), torch.from_numpy(db))
        return torch.from_numpy(ps)

    @staticmethod
    def backward(ctx, grad_out):
        dg, db = ctx.saved_tensors
        go = grad_out.to(torch.float64).reshape(-1, 1)
        return (go * dg).sum(0), (go * db).sum(0), None, None, None, None, None, None


def psucc(gamma, beta, costs, n, m, dtype="c64", flags=0, work=None):
    return QaoaPsucc.apply(gamma, beta, costs, n, m, dtype, flags, work)


def train_angles(costs: torch.Tensor, n: int, m: int, gamma0, beta0, steps: int = 200, lr: float = 0.01,
                 objective: str = "mean_log", dtype="c64", flags: int = 0, checkpoint: Optional[str] = None,
                 checkpoint_every: int = 20, log=None):
    """Adam on the shared angles to maximise mean log p_succ (or mean p_succ).

    Resumes from ``checkpoint`` (JSON: angles, Adam moments, step, trace) when it
    exists and writes it every ``checkpoint_every`` steps.  Returns (gamma, beta,
    trace) with trace = list of (step, objective)."""
    gamma = torch.tensor(np.asarray(gamma0, dtype=np.float64), requires_grad=True)
    beta = torch.tensor(np.asarray(beta0, dtype=np.float64), requires_grad=True)
    opt = torch.optim.Adam([gamma, beta], lr=lr)
    trace = []
    start = 0
    if checkpoint and os.path.exists(checkpoint):
        with open(checkpoint) as f:
            ck = json.load(f)
        with torch.no_grad():
            gamma.copy_(torch.tensor(ck["gamma"], dtype=torch.float64))
            beta.copy_(torch.tensor(ck["beta"], dtype=torch.float64))
        opt.load_state_dict(_opt_from_json(ck["adam"], opt))
        start, trace = ck["step"], [tuple(t) for t in ck["trace"]]
    B = int(costs.shape[0])
    work = (torch.empty((B, 1 << n), dtype=api.TORCH_DTYPE[api.dtype_code(dtype)], device="cuda"),
            torch.empty((B, 1 << n), dtype=api.TORCH_DTYPE[api.dtype_code(dtype)], device="cuda"))
    for step in range(start, steps):
        opt.zero_grad()
        p = psucc(gamma, beta, costs, n, m, dtype, flags, work)
        obj = torch.log(p).mean() if objective == "mean_log" else p.mean()
        (-obj).backward()
        opt.step()
        trace.append((step, float(obj.detach())))
        if log:
            log(step, float(obj.detach()))
        if checkpoint and ((step + 1) % checkpoint_every == 0 or step + 1 == steps):
            _save(checkpoint, gamma, beta, opt, step + 1, trace)
    return gamma.detach().numpy().copy(), beta.detach().numpy().copy(), trace


def _opt_to_json(opt):
    sd = opt.state_dict()
    state = {str(k): {kk: (vv.tolist() if torch.is_tensor(vv) else vv) for kk, vv in v.items()}
             for k, v in sd["state"].items()}
    return {"state": state, "param_groups": sd["param_groups"]}


def _opt_from_json(d, opt):
    sd = opt.state_dict()
    state = {int(k): {kk: torch.tensor(vv, dtype=torch.float64) if isinstance(vv, list) else
                      torch.tensor(vv, dtype=torch.float32) if kk == "step" else vv for kk, vv in v.items()}
             for k, v in d["state"].items()}
    return {"state": state, "param_groups": d["param_groups"] if d["param_groups"] else sd["param_groups"]}


def _save(path, gamma, beta, opt, step, trace):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump({"gamma": gamma.detach().tolist(), "beta": beta.detach().tolist(), "adam": _opt_to_json(opt),
                   "step": step, "trace": trace}, f)
    os.replace(tmp, path)
