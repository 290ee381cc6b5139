"""Angle training through torch.autograd with the adjoint gradient."""
import os

import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api, train  # noqa: E402


def _batch(n, B, tag):
    insts = [gen.satisfiable_instance(tag, n, 5, 8.0, i, oracle.count_solutions)[0] for i in range(B)]
    costs, _, _ = api.cost_table_batch(insts)
    return insts, costs


def test_autograd_matches_oracle_gradient():
    n, B, p = 14, 3, 3
    insts, costs = _batch(n, B, "ag")
    g0, b0 = gen.linear_ramp(p)
    gamma = torch.tensor(g0, requires_grad=True)
    beta = torch.tensor(b0, requires_grad=True)
    ps = train.psucc(gamma, beta, costs, n, insts[0].m, "c128")
    torch.log(ps).mean().backward()
    ref_g = np.zeros(p)
    ref_b = np.zeros(p)
    for inst in insts:
        cost, _, _ = oracle.cost_table(n, inst.var, inst.neg)
        rp, rdg, rdb = oracle.grad(n, cost, g0, b0)
        ref_g += rdg / rp / B
        ref_b += rdb / rp / B
    assert np.allclose(gamma.grad.numpy(), ref_g, rtol=1e-7, atol=1e-10)
    assert np.allclose(beta.grad.numpy(), ref_b, rtol=1e-7, atol=1e-10)


def test_adam_improves_mean_log_psucc_and_resumes(tmp_path):
    n, B, p = 16, 4, 3
    insts, costs = _batch(n, B, "adam")
    g0, b0 = gen.linear_ramp(p)
    g1, b1, trace = train.train_angles(costs, n, insts[0].m, g0, b0, steps=12, lr=0.05)
    assert trace[-1][1] > trace[0][1]
    ck = os.path.join(tmp_path, "ck.json")
    train.train_angles(costs, n, insts[0].m, g0, b0, steps=6, lr=0.05, checkpoint=ck, checkpoint_every=3)
    g2, b2, trace2 = train.train_angles(costs, n, insts[0].m, g0, b0, steps=12, lr=0.05, checkpoint=ck)
    assert len(trace2) == 12
    assert np.allclose(g1, g2, rtol=1e-6, atol=1e-9) and np.allclose(b1, b2, rtol=1e-6, atol=1e-9)
