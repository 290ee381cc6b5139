"""Host logic of angle training, without a GPU: the Adam state written to a
checkpoint (angles, moments, step count as JSON) restores an optimizer that
continues exactly as the uninterrupted one does, and the autograd function's
backward contracts the stored per-instance gradients with the incoming one."""
import json

import numpy as np
import torch

from paper_2401_02852_gb300 import train


def _grad(step, x):
    # a deterministic, step-dependent gradient (no randomness, no GPU)
    return torch.sin(x * (step + 1)) + 0.1 * step


def test_adam_state_round_trip_continues_identically(tmp_path):
    p = 3
    g0 = torch.tensor(np.linspace(-0.3, 0.2, p), dtype=torch.float64, requires_grad=True)
    b0 = torch.tensor(np.linspace(0.5, 0.1, p), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([g0, b0], lr=0.05)

    def step(o, g, b, s):
        o.zero_grad()
        g.grad = _grad(s, g.detach())
        b.grad = _grad(s, b.detach() + 1.0)
        o.step()

    for s in range(4):
        step(opt, g0, b0, s)
    path = str(tmp_path / "ck.json")
    train._save(path, g0, b0, opt, 4, [(s, 0.0) for s in range(4)])
    with open(path) as f:
        ck = json.load(f)
    assert ck["step"] == 4 and len(ck["trace"]) == 4

    g1 = torch.tensor(ck["gamma"], dtype=torch.float64, requires_grad=True)
    b1 = torch.tensor(ck["beta"], dtype=torch.float64, requires_grad=True)
    opt1 = torch.optim.Adam([g1, b1], lr=0.05)
    opt1.load_state_dict(train._opt_from_json(ck["adam"], opt1))
    for s in range(4, 9):
        step(opt, g0, b0, s)
        step(opt1, g1, b1, s)
    assert torch.equal(g0.detach(), g1.detach()) and torch.equal(b0.detach(), b1.detach())


def test_backward_contracts_per_instance_gradients():
    dg = torch.tensor([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]], dtype=torch.float64)
    db = torch.tensor([[0.5, -1.0], [0.0, 2.0], [1.0, 1.0]], dtype=torch.float64)

    class Ctx:
        saved_tensors = (dg, db)

    go = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    out = train.QaoaPsucc.backward(Ctx(), go)
    assert torch.allclose(out[0], (go[:, None] * dg).sum(0)) and torch.allclose(out[1], (go[:, None] * db).sum(0))
    assert all(o is None for o in out[2:])
