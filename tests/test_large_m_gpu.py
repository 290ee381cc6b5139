"""Clause counts beyond the kernel-parameter list (up to 8191: the densities of
the paper's protocol, r_hat_k n at k = 9, 10 and n <= 19) against the oracle.

* cost tables bit-exact: single, half, batched with mixed m around the chunk
  boundary (1024 records), and the overflow report (exact max C past 255);
* evolutions and gradients with m > 255: the phase tables stop at the uint8
  range, which every C(x) of an accepted table is in;
* the serving loop (packed and single launches) on such instances;
* the protocol's plumbing at a small size: training objective, evaluation
  and fits.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api, protocol  # noqa: E402
from paper_2401_02852_gb300._lib import load  # noqa: E402


def _inst(tag, n, k, m, idx=0):
    var, neg = gen.draw_clauses_keys(n, k, m, gen.rng_for(tag, n, k, m, idx))
    return gen.Instance(n=n, k=k, var=var, neg=neg)


def _sat_protocol_inst(tag, n, k):
    for a in range(200):
        inst = gen.protocol_instance(tag, n, k, 0, a)
        cost, sol, _ = oracle.cost_table(n, inst.var, inst.neg)
        if sol:
            return inst, cost
    raise RuntimeError("no satisfiable instance")


@pytest.mark.parametrize("n,k,m", [(12, 9, 2121), (13, 6, 1024), (13, 6, 1025), (14, 10, 4960), (16, 9, 2830),
                                   (17, 10, 8191), (19, 9, 3360)])
def test_cost_table_large_m_bit_exact(n, k, m):
    inst = _inst("ctm", n, k, m)
    ref, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
    assert mx <= 255
    cost, gsol, gmx = api.cost_table(inst)
    assert np.array_equal(cost.cpu().numpy(), ref.astype(np.uint8))
    assert (gsol, gmx) == (sol, mx)
    half, hsol, hmx = api.cost_table_half(inst)
    assert np.array_equal(half.cpu().numpy(), ref[: 1 << (n - 1)].astype(np.uint8))
    assert (hsol, hmx) == (sol, mx)


def test_cost_table_batch_mixed_m():
    n = 14
    ms = [0, 700, 1023, 1024, 1025, 3000, 8191, 16]
    insts = [_inst("ctbm", n, 7, m, i) for i, m in enumerate(ms)]
    costs, sols, mxs = api.cost_table_batch(insts)
    for i, inst in enumerate(insts):
        ref, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
        assert np.array_equal(costs[i].cpu().numpy(), ref.astype(np.uint8)), ms[i]
        assert (int(sols[i]), int(mxs[i])) == (sol, mx)


def test_overflow_with_long_clause_list_reports_exact_stats():
    """5000 two-literal clauses: counts near 2500, past 255 and past 10 bit
    planes; the call fails with the exact max and solution count."""
    n = 9
    inst = _inst("ovfm", n, 2, 5000)
    ref, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
    assert mx > 1023
    ci = api._Inst(inst)
    out = torch.empty(1 << n, dtype=torch.uint8, device="cuda")
    ns, gm = ctypes.c_uint64(), ctypes.c_uint32()
    rc = load().naesat_cost_table(ctypes.byref(ci.s), api._ptr(out), ctypes.byref(ns), ctypes.byref(gm),
                                  api._stream(None))
    assert rc == -2 and ns.value == sol and gm.value == mx
    assert np.array_equal(out.cpu().numpy(), (ref % 256).astype(np.uint8))


@pytest.mark.parametrize("n,k", [(12, 9), (15, 9), (13, 10)])
def test_evolve_large_m_matches_oracle(n, k):
    inst, ref_cost = _sat_protocol_inst(f"evm-{n}", n, k)
    assert inst.m > 255
    g, b = gen.linear_ramp(6, scale=0.3)
    cost, _, _ = api.cost_table(inst)
    psi = oracle.evolve(n, ref_cost, g, b)
    ref_ps, _ = oracle.success_prob(n, ref_cost, psi)
    state, ps, norm = api.evolve(n, cost, inst.m, g, b, "c128")
    assert abs(ps - ref_ps) <= 1e-10 * ref_ps and abs(norm - 1) < 1e-12
    assert np.max(np.abs(state.cpu().numpy() - psi)) < 1e-13
    state, ps, norm = api.evolve(n, cost, inst.m, g, b, "c64")
    assert abs(ps - ref_ps) <= 1e-4 * ref_ps and abs(norm - 1) < 1e-6


def test_halved_state_large_m():
    """The halved state with a long clause list gives the full state's p_succ
    and amplitudes (global-flip symmetry, C(not x) = C(x))."""
    from paper_2401_02852_gb300._lib import Z2_HALF
    n = 17
    inst, ref_cost = _sat_protocol_inst("z2m", n, 9)
    g, b = gen.linear_ramp(5, scale=0.3)
    cost = api.cost_table(inst)[0]
    half = api.cost_table_half(inst)[0]
    full, ps, _ = api.evolve(n, cost, inst.m, g, b, "c128")
    st_h, ps_h, nm_h = api.evolve(n, half, inst.m, g, b, "c128", flags=Z2_HALF)
    assert abs(ps_h - ps) <= 1e-12 * ps and abs(nm_h - 1) < 1e-12
    assert float((st_h - full[: 1 << (n - 1)]).abs().max()) < 1e-13


@pytest.mark.parametrize("n,dtype", [(12, "c128"), (15, "c128"), (15, "c64")])
def test_grad_large_m_matches_oracle(n, dtype):
    inst, ref_cost = _sat_protocol_inst(f"grm-{n}", n, 9)
    p = 3
    g, b = gen.linear_ramp(p, scale=0.3)
    cost, _, _ = api.cost_table(inst)
    ps, dg, db = api.grad(n, cost, inst.m, g, b, dtype)
    rps, rdg, rdb = oracle.grad(n, ref_cost, g, b)
    scale = max(np.max(np.abs(rdg)), np.max(np.abs(rdb)))
    tol = 1e-8 if dtype == "c128" else 1e-6 * (1 + n * p)
    assert abs(ps - rps) <= (1e-10 if dtype == "c128" else 1e-4) * rps
    assert np.max(np.abs(dg - rdg)) <= tol * scale and np.max(np.abs(db - rdb)) <= tol * scale


def test_serving_large_m():
    from paper_2401_02852_gb300.serve import Server

    reqs = [_sat_protocol_inst(f"srvm-{n}", n, 9) for n in (12, 16)]
    g, b = gen.linear_ramp(4, scale=0.3)
    with Server("c64") as s:
        res = [s.wait(s.submit(inst, g, b)) for inst, _ in reqs]
    for (inst, ref_cost), r in zip(reqs, res):
        ref_ps, _ = oracle.success_prob(inst.n, ref_cost, oracle.evolve(inst.n, ref_cost, g, b))
        assert r.status == 0 and r.n_sol == int(np.sum(ref_cost == 0)) and r.max_cost == int(ref_cost.max())
        assert abs(r.p_succ - ref_ps) <= 1e-4 * ref_ps


def test_protocol_training_objective_and_evaluation():
    """The training objective at the initial angles is the mean oracle p_succ of
    the training instances; the evaluation's instances are satisfiable, its
    p_hat is the mean of per-instance p_succ the oracle reproduces, and every
    running time is a positive draw count."""
    k, p, t = 5, 2, 6
    g, b, trace = protocol.train_fixed_angles(k, p, t=t, epochs=2, lr=1e-3)
    insts = [gen.protocol_instance("protocol-train", 12, k, i) for i in range(t)]
    want = np.mean([oracle.success_prob(12, c, oracle.evolve(12, c, np.full(p, -0.01), np.full(p, 0.01)))[0]
                    for c in (oracle.cost_table(12, i.var, i.neg)[0] for i in insts)])
    assert trace[0][1] == pytest.approx(want, rel=1e-10)
    assert np.all(np.abs(g + 0.01) <= 3e-3) and np.all(np.abs(b - 0.01) <= 3e-3)  # two Adam steps of about lr
    ev = protocol.evaluate(k, {p: (g, b)}, ns=(12, 14), count=10, tag="protocol-test")
    sat, _ = protocol.satisfiable_batch("protocol-test-k5", 14, k, 10)
    ps = []
    for inst in sat:
        c, sol, _ = oracle.cost_table(14, inst.var, inst.neg)
        assert sol > 0
        ps.append(oracle.success_prob(14, c, oracle.evolve(14, c, g, b))[0])
    assert ev["points"][(p, 14)]["mean_psucc"] == pytest.approx(np.mean(ps), rel=1e-4)
    assert ev["points"][(p, 12)]["median_running_time"] >= 1
    assert ev["points"][(p, 14)]["censored_running_times"] == 0
    res = protocol.run_protocol(ks=(5,), ps=(1, 2), ns=range(12, 15), t=4, epochs=2, count=8)
    ex = res["by_k"]["5"]["exponents"]
    assert set(ex["by_p"]) == {"1", "2"} and ex["random_assignment"]["nat"] > 0
    assert "power_law_bits" in ex


def test_protocol_k9_reproduces_the_papers_power_law():
    """The paper's main-text ensemble (k = 9, 2500 satisfiable instances per
    n = 12..19, nine depths, angles trained at n = 12 with lr 0.01): the
    median-running-time exponents in bits follow a p^b close to the paper's
    table (a = 0.686, b = -0.222), fall with p, and agree with the p_hat
    exponents to within a fifth at every depth."""
    ps = (1, 2, 4, 8, 16, 20, 24, 28, 32)
    res = protocol.run_protocol(ks=(9,), ps=ps, count=2500)
    ex = res["by_k"]["9"]["exponents"]
    a, b = ex["power_law_bits"]
    pa, pb = protocol.PAPER_POWER_LAW[9]
    assert abs(a - pa) < 0.05 and abs(b - pb) < 0.06, (a, b)
    ct = [ex["by_p"][str(p)]["C_tilde_bits"] for p in ps]
    assert ct[0] > ct[4] > ct[-1] > 0
    assert max(ex["by_p"][str(p)]["relative_error"] for p in ps) < 0.25
    assert ct[0] < ex["random_assignment"]["bits"]
