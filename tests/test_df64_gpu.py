"""complex128 evolutions in double-float arithmetic (QAOA_DF64) against the
FP64 oracle and the native FP64 path.

Tolerance, from the arithmetic: a double-float multiply-add is exact to about
2^-46 of its operands (the dropped lo x lo product and the final
renormalisation), and an amplitude goes through at most n p butterfly stages
plus p phase products, so |psi_df - psi| <= 2e-12 (1 + n p) max|psi| (a linear
bound with margin); p_succ agrees within 1e-10 relative, the complex128
requirement.
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
from paper_2401_02852_gb300._lib import DF64, Z2_HALF, QaoaError  # noqa: E402


# n <= 12: the one-CTA kernel in double-float; larger n: the passes
@pytest.mark.parametrize("n,p,sign", [(6, 2, 1), (8, 5, -1), (12, 5, 1), (14, 1, 1), (17, 3, 1), (20, 6, -1),
                                      (22, 4, 1)])
def test_df64_matches_oracle(n, p, sign):
    inst, _ = gen.satisfiable_instance("df64", n, 5, 8.0, n, oracle.count_solutions)
    cost_o, _, _ = oracle.cost_table(n, inst.var, inst.neg)
    g, b = gen.linear_ramp(p)
    psi_o = oracle.evolve(n, cost_o, g, b, sign)
    ps_o, nm_o = oracle.success_prob(n, cost_o, psi_o)
    cost = api.cost_table(inst)[0]
    flags = DF64 | (0 if sign == 1 else api.MIXER_RX2B)
    st, ps, nm = api.evolve(n, cost, inst.m, g, b, "c128", flags=flags)
    psi = st.cpu().numpy()
    tol = 2e-12 * (1 + n * p) * np.max(np.abs(psi_o))
    assert np.max(np.abs(psi - psi_o)) <= tol
    assert abs(ps - ps_o) <= 1e-10 * ps_o and abs(nm - nm_o) <= 1e-10


def test_df64_matches_fp64_and_batch():
    n, p, B = 24, 10, 3
    insts = [gen.raw_instance("df64-b", n, 5, 8.0, i) for i in range(B)]
    costs, sols, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(p)
    st64, ps64, _ = api.evolve_batch(n, costs, insts[0].m, g, b, "c128")
    stdf, psdf, nmdf = api.evolve_batch(n, costs, insts[0].m, g, b, "c128", flags=DF64)
    for i in range(B):
        tol = 2e-12 * (1 + n * p) * float(st64[i].abs().max())
        assert float((stdf[i] - st64[i]).abs().max()) <= tol
        if sols[i]:
            assert abs(psdf[i] - ps64[i]) <= 1e-10 * ps64[i]
        assert abs(nmdf[i] - 1) < 1e-10
    one, _, _ = api.evolve(n, costs[1].contiguous(), insts[1].m, g, b, "c128", flags=DF64)
    assert torch.equal(one, stdf[1])


def test_df64_small_batch_matches_fp64():
    """The batched one-CTA path (100 instances of n = 12, the complex128 batch
    workload's shape) in double-float against FP64."""
    n, p, B = 12, 5, 100
    insts = [gen.raw_instance("df64-small", n, 3, 2.0, i) for i in range(B)]
    costs, sols, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(p)
    st64, ps64, _ = api.evolve_batch(n, costs, insts[0].m, g, b, "c128")
    stdf, psdf, nmdf = api.evolve_batch(n, costs, insts[0].m, g, b, "c128", flags=DF64)
    assert float((stdf - st64).abs().max()) <= 2e-12 * (1 + n * p) * float(st64.abs().max())
    for i in range(B):
        if sols[i]:
            assert abs(psdf[i] - ps64[i]) <= 1e-10 * ps64[i]
        assert abs(nmdf[i] - 1) < 1e-10


def test_df64_serving_matches_direct_evolutions():
    """A complex128 server in double-float arithmetic (packed small requests
    and single large ones) gives the direct QAOA_DF64 evolution's numbers."""
    from paper_2401_02852_gb300.serve import Server
    reqs = [(gen.raw_instance("df64-srv", n, 5, 8.0, i), n) for i, n in enumerate((10, 12, 15, 18))]
    g, b = gen.linear_ramp(4)
    with Server("c128", flags=DF64) as s:
        res = [s.wait(s.submit(inst, g, b)) for inst, _ in reqs]
    for (inst, n), r in zip(reqs, res):
        cost = api.cost_table(inst)[0]
        _, ps, nm = api.evolve(n, cost, inst.m, g, b, "c128", flags=DF64)
        _, ps64, _ = api.evolve(n, cost, inst.m, g, b, "c128")
        assert r.status == 0 and abs(r.norm - nm) <= 1e-13
        assert abs(r.p_succ - ps) <= 1e-13 * max(ps, 1e-300) and abs(r.p_succ - ps64) <= 1e-10 * max(ps64, 1e-300)


def test_df64_p0_is_plus_state():
    n = 16
    inst = gen.raw_instance("df64-p0", n, 5, 8.0, 0)
    cost = api.cost_table(inst)[0]
    st, ps, nm = api.evolve(n, cost, inst.m, [], [], "c128", flags=DF64)
    assert torch.allclose(st, torch.full_like(st, 2.0 ** (-n / 2)), rtol=0, atol=1e-15)
    assert abs(nm - 1) < 1e-12


def test_df64_rejects_other_modes():
    n = 16
    inst = gen.raw_instance("df64-rej", n, 5, 8.0, 0)
    cost = api.cost_table(inst)[0]
    g, b = gen.linear_ramp(2)
    with pytest.raises(QaoaError):
        api.evolve(n, cost, inst.m, g, b, "c64", flags=DF64)
    half = api.cost_table_half(inst)[0]
    with pytest.raises(QaoaError):
        api.evolve(n, half, inst.m, g, b, "c128", flags=DF64 | Z2_HALF)
    with pytest.raises(QaoaError):
        api.grad(n, cost, inst.m, g, b, "c128", flags=DF64)
    from paper_2401_02852_gb300.serve import Server
    with pytest.raises(QaoaError):
        Server("c64", flags=DF64)
    with pytest.raises(QaoaError):
        Server("c128", flags=DF64 | Z2_HALF)


@pytest.mark.slow
def test_df64_full_size_n30():
    n, p = 30, 10
    inst, _ = gen.satisfiable_instance("bench-n30", n, 5, 8.0, 0, lambda x: api.cost_table(x)[1])
    cost = api.cost_table(inst)[0]
    g, b = gen.linear_ramp(p)
    st64, ps64, _ = api.evolve(n, cost, inst.m, g, b, "c128")
    stdf = torch.empty_like(st64)
    _, psdf, nmdf = api.evolve(n, cost, inst.m, g, b, "c128", flags=DF64, out=stdf)
    assert abs(psdf - ps64) <= 1e-10 * ps64 and abs(nmdf - 1) < 1e-10
    xs = torch.from_numpy(gen.rng_for("df64-n30", 0).integers(0, 1 << n, size=100000).astype(np.int64)).cuda()
    tol = 2e-12 * (1 + n * p) * float(st64[xs].abs().max())
    assert float((stdf[xs] - st64[xs]).abs().max()) <= tol
    del st64, stdf
    torch.cuda.empty_cache()
