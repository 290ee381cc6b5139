"""Parity at the configured workload sizes, against the FP64 oracle.

* 100 satisfiable NAE-3-SAT instances, n = 12, m = 24, p = 5, complex128,
  one batched launch: cost tables bit-exact, p_succ within 1e-10 relative.
* The gradient workload's shape (NAE-5-SAT, n = 22, m = 176, p = 20): the
  batched complex64 adjoint gradient of a few instances against the oracle's
  stored-state gradient (tolerance 1e-6 (1 + n p) of max |g|), complex128 within 1e-8.
"""
import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api  # noqa: E402


def test_batch_of_100_small_instances_c128():
    n, k, r, p = 12, 3, 2.0, 5
    insts = [gen.satisfiable_instance("cfg1", n, k, r, i, oracle.count_solutions)[0] for i in range(100)]
    costs, sols, mxs = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(p)
    states, ps, nm = api.evolve_batch(n, costs, insts[0].m, g, b, "c128")
    host = costs.cpu().numpy()
    for i, inst in enumerate(insts):
        ref, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
        assert np.array_equal(host[i], ref.astype(np.uint8))
        assert (int(sols[i]), int(mxs[i])) == (sol, mx)
        rps, rnm = oracle.success_prob(n, ref, oracle.evolve(n, ref, g, b))
        assert abs(ps[i] - rps) <= 1e-10 * rps
        assert abs(nm[i] - 1) < 1e-12


@pytest.mark.slow
def test_gradient_workload_shape_against_oracle():
    n, p, B = 22, 20, 3
    insts = [gen.satisfiable_instance("cfg4", n, 5, 8.0, i, lambda x: api.cost_table(x)[1])[0] for i in range(B)]
    costs, _, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(p)
    ps, dg, db = api.grad_batch(n, costs, insts[0].m, g, b, "c64")
    ref = oracle.cost_table(n, insts[0].var, insts[0].neg)[0]
    rps, rdg, rdb = oracle.grad(n, ref, g, b)
    scale = max(np.max(np.abs(rdg)), np.max(np.abs(rdb)))
    assert abs(ps[0] - rps) <= 1e-4 * rps
    tol = 1e-6 * (1 + n * p) * scale
    assert np.max(np.abs(dg[0] - rdg)) <= tol
    assert np.max(np.abs(db[0] - rdb)) <= tol
    p1, g1, b1 = api.grad(n, costs[0].contiguous(), insts[0].m, g, b, "c128")
    assert abs(p1 - rps) <= 1e-10 * rps
    assert np.max(np.abs(g1 - rdg)) <= 1e-8 * scale and np.max(np.abs(b1 - rdb)) <= 1e-8 * scale
