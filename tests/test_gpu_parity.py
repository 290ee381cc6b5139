"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here; each follows from the rounding of the arithmetic):
  * cost table, solution count, max C: bit-exact;
  * complex128 path: p_succ relative error <= 1e-10, amplitudes within 1e-13;
  * complex64 path: p_succ relative error <= 1e-4, norm within 1e-6, amplitudes
    within 1e-6 (1 + n p) max|psi| (FP32 rounding per butterfly, n p butterflies);
    a uniform state (gamma = 0 or no clauses) rounds every amplitude the same
    way, so its norm drifts coherently: 1e-5 there (2 u per stage, n p stages);
  * the reduction of a given complex64 state: within 8 u = 4.8e-7 relative
    (pairwise FP32 sums of a thread's 32 terms, FP64 above);
  * gradients: complex128 within 1e-8 of the oracle (relative to max |g|),
    complex64 within 1e-6 (1 + n p) (the amplitude bound's factor).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api  # noqa: E402
from paper_2401_02852_gb300._lib import QaoaError  # noqa: E402

C128_PS_TOL = 1e-10
C64_PS_TOL = 1e-4


def _inst(tag, n, k, m, idx=0):
    var, neg = gen.draw_clauses(n, k, m, gen.rng_for(tag, n, k, m, idx))
    return gen.Instance(n=n, k=k, var=var, neg=neg)


def _sat_inst(tag, n, k, m):
    """First satisfiable draw (k = 1 clauses are always violated, so those cases use m = 0)."""
    for idx in range(2000):
        inst = _inst(tag, n, k, m, idx)
        cost, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
        if sol:
            return inst, cost
    raise RuntimeError("no satisfiable instance")


# ---------------------------------------------------------------------------
# cost table


@pytest.mark.parametrize("n,k,m", [(1, 1, 3), (3, 3, 4), (4, 2, 7), (5, 3, 16), (6, 5, 17), (9, 3, 0),
                                   (12, 3, 24), (13, 7, 100), (17, 5, 136), (20, 4, 255), (24, 5, 192),
                                   (10, 10, 33), (11, 2, 300)])
def test_cost_table_bit_exact(n, k, m):
    inst = _inst("ct", n, k, m)
    ref, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
    if mx > 255:
        with pytest.raises(QaoaError):
            api.cost_table(inst)
        return
    cost, gsol, gmx = api.cost_table(inst)
    assert np.array_equal(cost.cpu().numpy(), ref.astype(np.uint8))
    assert (gsol, gmx) == (sol, mx)


def test_cost_table_overflow_reports_exact_stats():
    """m = 300 two-literal clauses give counts above 255: ERANGE, exact max and count."""
    inst = _inst("ovf", 8, 2, 600)
    ref, sol, mx = oracle.cost_table(8, inst.var, inst.neg)
    assert mx > 255
    import ctypes

    from paper_2401_02852_gb300._lib import load
    ci = api._Inst(inst)
    out = torch.empty(1 << 8, dtype=torch.uint8, device="cuda")
    ns, gm = ctypes.c_uint64(), ctypes.c_uint32()
    rc = load().naesat_cost_table(ctypes.byref(ci.s), api._ptr(out), ctypes.byref(ns), ctypes.byref(gm),
                                  api._stream(None))
    assert rc == -2 and ns.value == sol and gm.value == mx
    assert np.array_equal(out.cpu().numpy(), (ref % 256).astype(np.uint8))


def test_hand_tables_on_gpu():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_cost_tables.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        var = np.array(c["var"], dtype=np.int32)
        inst = gen.Instance(n=c["n"], k=var.shape[1], var=var, neg=np.array(c["neg"], dtype=np.uint8))
        cost, sol, _ = api.cost_table(inst)
        assert cost.cpu().tolist() == c["cost"], c["name"]
        assert sol == c["n_sol"]


def test_cost_table_batch_matches_single():
    insts = [_inst("ctb", 14, 5, 112, i) for i in range(7)]
    costs, sols, mxs = api.cost_table_batch(insts)
    for i, inst in enumerate(insts):
        ref, sol, mx = oracle.cost_table(14, inst.var, inst.neg)
        assert np.array_equal(costs[i].cpu().numpy(), ref.astype(np.uint8))
        assert (int(sols[i]), int(mxs[i])) == (sol, mx)


def test_invalid_instances_rejected():
    bad = gen.Instance(n=4, k=2, var=np.array([[0, 0]], dtype=np.int32), neg=np.zeros((1, 2), np.uint8))
    with pytest.raises(QaoaError):
        api.cost_table(bad)
    bad = gen.Instance(n=4, k=2, var=np.array([[0, 4]], dtype=np.int32), neg=np.zeros((1, 2), np.uint8))
    with pytest.raises(QaoaError):
        api.cost_table(bad)
    bad = gen.Instance(n=33, k=2, var=np.array([[0, 1]], dtype=np.int32), neg=np.zeros((1, 2), np.uint8))
    with pytest.raises(QaoaError):
        api.cost_table(bad)


# ---------------------------------------------------------------------------
# evolution


def _angles(p, kind):
    if kind == "ramp":
        return gen.linear_ramp(p)
    rng = gen.rng_for("angles", p, {"rand": 1, "steep": 2}[kind])
    g = rng.uniform(-2.0, 2.0, p)
    b = rng.uniform(-1.5, 1.5, p)
    if kind == "steep":  # |tan beta| > 1 exercises the second butterfly form
        b = np.where(np.arange(p) % 2 == 0, 1.2, -1.35)
    return g, b


EVOLVE_CASES = [(1, 1, 0, 2), (2, 2, 3, 1), (5, 3, 10, 3), (12, 3, 24, 5), (13, 3, 26, 3), (14, 5, 112, 2),
                (16, 5, 128, 4), (20, 5, 160, 3), (22, 4, 100, 2)]


@pytest.mark.parametrize("n,k,m,p", EVOLVE_CASES)
@pytest.mark.parametrize("kind", ["ramp", "steep"])
def test_evolve_c128_matches_oracle(n, k, m, p, kind):
    inst, ref_cost = _sat_inst("ev", n, k, m)
    g, b = _angles(p, kind)
    cost, _, _ = api.cost_table(inst)
    state, ps, norm = api.evolve(n, cost, inst.m, g, b, "c128")
    psi = oracle.evolve(n, ref_cost, g, b)
    ref_ps, _ = oracle.success_prob(n, ref_cost, psi)
    assert abs(ps - ref_ps) <= C128_PS_TOL * abs(ref_ps) + 1e-300
    assert abs(norm - 1.0) < 1e-12
    got = state.cpu().numpy()
    assert np.max(np.abs(got - psi)) < 1e-13


@pytest.mark.parametrize("n,k,m,p", EVOLVE_CASES)
@pytest.mark.parametrize("sign", [0, 1])
def test_evolve_c64_matches_oracle(n, k, m, p, sign):
    inst, ref_cost = _sat_inst("ev64", n, k, m)
    g, b = _angles(p, "ramp" if p % 2 else "rand")
    cost, _, _ = api.cost_table(inst)
    state, ps, norm = api.evolve(n, cost, inst.m, g, b, "c64", flags=sign)
    psi = oracle.evolve(n, ref_cost, g, b, -1 if sign else 1)
    ref_ps, _ = oracle.success_prob(n, ref_cost, psi)
    assert abs(ps - ref_ps) <= C64_PS_TOL * abs(ref_ps)
    assert abs(norm - 1.0) < 1e-6
    got = state.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - psi)) <= 1e-6 * (1 + n * p) * np.max(np.abs(psi))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_p0_and_random_assignment_theorem(dtype):
    """p = 0, gamma = 0 or beta = 0: p_succ = #sol / 2^n (Appendix B)."""
    n = 17
    inst, ref_cost = _sat_inst("thm", n, 5, 136)
    sol = int((ref_cost == 0).sum())
    cost, gsol, _ = api.cost_table(inst)
    assert gsol == sol
    tol = 1e-12 if dtype == "c128" else 1e-5  # uniform state: coherent FP32 rounding
    for g, b in [([], []), (np.zeros(3), np.array([0.3, 1.2, -0.4])), (np.array([0.5, -1.0]), np.zeros(2))]:
        _, ps, norm = api.evolve(n, cost, inst.m, g, b, dtype)
        assert abs(ps - sol / 2 ** n) <= tol * sol / 2 ** n
        assert abs(norm - 1) < tol


def test_empty_instance_all_solutions():
    """m = 0: every x is a solution, so p_succ = norm = 1 for any angles."""
    inst = gen.Instance(n=15, k=3, var=np.zeros((0, 3), np.int32), neg=np.zeros((0, 3), np.uint8))
    cost, sol, mx = api.cost_table(inst)
    assert sol == 2 ** 15 and mx == 0
    _, ps, norm = api.evolve(15, cost, 0, *gen.linear_ramp(3), "c64")
    assert abs(ps - 1) < 1e-5 and abs(norm - 1) < 1e-5


def test_success_prob_standalone():
    n = 19
    inst, ref_cost = _sat_inst("sp", n, 5, 152)
    g, b = gen.linear_ramp(4)
    cost, _, _ = api.cost_table(inst)
    for dtype, tol in (("c128", 1e-12), ("c64", 8 * 2.0 ** -24)):
        state, ps, norm = api.evolve(n, cost, inst.m, g, b, dtype)
        ps2, norm2 = api.success_prob(n, cost, state)
        ref = oracle.success_prob(n, ref_cost, state.cpu().numpy().astype(np.complex128))
        assert abs(ps2 - ref[0]) <= tol * ref[0] and abs(norm2 - ref[1]) <= tol * ref[1]
        # the fused reduction of the last pass: the same bound against the oracle
        assert abs(ps - ref[0]) <= tol * ref[0] and abs(norm - ref[1]) <= tol * ref[1]


@pytest.mark.parametrize("n", [12, 16])
def test_evolve_batch_matches_single(n):
    insts = [_inst("evb", n, 5, 8 * n, i) for i in range(5)]
    costs, _, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(5)
    states, ps, nm = api.evolve_batch(n, costs, 8 * n, g, b, "c64")
    for i in range(5):
        st, p1, n1 = api.evolve(n, costs[i].contiguous(), 8 * n, g, b, "c64")
        assert np.array_equal(states[i].cpu().numpy(), st.cpu().numpy())
        assert ps[i] == p1 and nm[i] == n1


def test_global_flip_symmetry_of_gpu_state():
    n = 21
    inst, _ = _sat_inst("flipgpu", n, 5, 168)
    cost, _, _ = api.cost_table(inst)
    state, _, _ = api.evolve(n, cost, inst.m, *gen.linear_ramp(3), "c128")
    s = state.cpu().numpy()
    x = np.arange(1 << n)
    assert np.max(np.abs(s - s[(~x) & ((1 << n) - 1)])) < 1e-15


# ---------------------------------------------------------------------------
# gradients


# n = 18: the high group is partial with 6 bits (runtime mask); n = 14, 15, 20,
# 21, 22: the last group's bits are within the load mapping's registers (no
# exchange); n = 20..22 also run a full 7- or 8-bit group
@pytest.mark.parametrize("n,dtype", [(9, "c128"), (9, "c64"), (14, "c128"), (15, "c64"), (18, "c128"), (18, "c64"),
                                     (20, "c64"), (21, "c128"), (21, "c64"), (22, "c64")])
@pytest.mark.parametrize("sign", [0, 1])
def test_grad_matches_oracle(n, dtype, sign):
    inst, ref_cost = _sat_inst("gr", n, 5, 8 * n)  # the configured gradient workload family (k = 5, r = 8)
    p = 4
    g, b = gen.linear_ramp(p)
    cost, _, _ = api.cost_table(inst)
    ps, dg, db = api.grad(n, cost, inst.m, g, b, dtype, flags=sign)
    rps, rdg, rdb = oracle.grad(n, ref_cost, g, b, -1 if sign else 1)
    scale = max(np.max(np.abs(rdg)), np.max(np.abs(rdb)))
    tol = 1e-8 if dtype == "c128" else 1e-6 * (1 + n * p)
    assert abs(ps - rps) <= (1e-10 if dtype == "c128" else 1e-4) * rps
    assert np.max(np.abs(dg - rdg)) <= tol * scale
    assert np.max(np.abs(db - rdb)) <= tol * scale


def test_grad_central_differences_on_gpu():
    n, p = 16, 3
    inst, _ = _sat_inst("grfd", n, 5, 128)
    cost, _, _ = api.cost_table(inst)
    g, b = gen.linear_ramp(p)
    _, dg, db = api.grad(n, cost, inst.m, g, b, "c128")
    h = 1e-4
    f = lambda gg, bb: api.evolve(n, cost, inst.m, gg, bb, "c128")[1]
    for l in range(p):
        e = np.zeros(p)
        e[l] = h
        fd_g = (f(g + e, b) - f(g - e, b)) / (2 * h)
        fd_b = (f(g, b + e) - f(g, b - e)) / (2 * h)
        assert abs(fd_g - dg[l]) < 1e-6 * max(1e-3, abs(fd_g)) + 1e-9
        assert abs(fd_b - db[l]) < 1e-6 * max(1e-3, abs(fd_b)) + 1e-9


def test_grad_batch_matches_single():
    n, p = 15, 3
    insts = [_inst("grb", n, 5, 120, i) for i in range(3)]
    costs, _, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(p)
    ps, dg, db = api.grad_batch(n, costs, 120, g, b, "c64")
    for i in range(3):
        p1, g1, b1 = api.grad(n, costs[i].contiguous(), 120, g, b, "c64")
        assert abs(ps[i] - p1) <= 1e-6 * abs(p1) + 1e-30
        assert np.allclose(dg[i], g1, rtol=1e-5, atol=1e-9) and np.allclose(db[i], b1, rtol=1e-5, atol=1e-9)


# ---------------------------------------------------------------------------
# full size (n = 30, the precision-study workload): sampled checks


@pytest.mark.slow
def test_full_size_n30_sampled():
    n, k, r, p = 30, 5, 8.0, 10
    inst, _ = gen.satisfiable_instance("full30", n, k, r, 0, lambda x: api.cost_table(x)[1])
    cost, sol, mx = api.cost_table(inst)
    assert sol > 0
    # sampled entries against the oracle's per-x definition
    xs = gen.rng_for("full30-xs", 0).integers(0, 1 << n, size=20000, dtype=np.uint64)
    ref = oracle.cost_samples(inst.var, inst.neg, xs)
    got = cost[torch.from_numpy(xs.astype(np.int64)).cuda()].cpu().numpy()
    assert np.array_equal(got, ref.astype(np.uint8))
    # exact clause-count identity over all 2^30 entries, and the flip symmetry on samples
    assert int(cost.sum(dtype=torch.int64).item()) == inst.m * 2 ** (n - k + 1)
    flip = torch.from_numpy(((~xs) & np.uint64((1 << n) - 1)).astype(np.int64)).cuda()
    assert torch.equal(cost[flip], cost[torch.from_numpy(xs.astype(np.int64)).cuda()])
    g, b = gen.linear_ramp(p)
    st64, ps64, nm64 = api.evolve(n, cost, inst.m, g, b, "c64")
    assert abs(nm64 - 1) < 1e-6
    idx = torch.from_numpy(xs.astype(np.int64)).cuda()
    assert torch.allclose(st64[idx], st64[flip], rtol=0, atol=1e-9)
    del st64
    torch.cuda.empty_cache()
    st128, ps128, nm128 = api.evolve(n, cost, inst.m, g, b, "c128")
    assert abs(nm128 - 1) < 1e-12
    assert abs(ps64 - ps128) <= C64_PS_TOL * ps128
    del st128
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_max_size_n32_sampled():
    """n = 32, the largest size (m = 256, the sweep's top point): sampled cost
    entries against the oracle, the clause-count identity over all 2^32 entries,
    a complex64 evolution (norm, flip symmetry) and the halved state's p_succ
    against the full one."""
    n, k, r, p = 32, 5, 8.0, 2
    inst, _ = gen.satisfiable_instance("full32", n, k, r, 0, lambda x: api.cost_table(x)[1])
    assert inst.m == 256
    cost, sol, mx = api.cost_table(inst)
    assert sol > 0
    assert mx <= 255  # a count of 256 would need every clause violated at one x
    xs = gen.rng_for("full32-xs", 0).integers(0, 1 << n, size=20000, dtype=np.uint64)
    ref = oracle.cost_samples(inst.var, inst.neg, xs)
    idx = torch.from_numpy(xs.astype(np.int64)).cuda()
    assert np.array_equal(cost[idx].cpu().numpy(), ref.astype(np.uint8))
    assert int(cost.sum(dtype=torch.int64).item()) == inst.m * 2 ** (n - k + 1)
    g, b = gen.linear_ramp(p)
    st, ps, nm = api.evolve(n, cost, inst.m, g, b, "c64")
    assert abs(nm - 1) < 1e-6
    flip = torch.from_numpy(((~xs) & np.uint64((1 << n) - 1)).astype(np.int64)).cuda()
    assert torch.allclose(st[idx], st[flip], rtol=0, atol=1e-9)
    del st
    torch.cuda.empty_cache()
    from paper_2401_02852_gb300._lib import Z2_HALF
    half = api.cost_table_half(inst)[0]
    assert torch.equal(half[:1 << 20], cost[:1 << 20])
    del cost
    torch.cuda.empty_cache()
    _, ps_h, nm_h = api.evolve(n, half, inst.m, g, b, "c64", flags=Z2_HALF)
    assert abs(nm_h - 1) < 1e-6
    assert abs(ps_h - ps) <= C64_PS_TOL * ps
    torch.cuda.empty_cache()
