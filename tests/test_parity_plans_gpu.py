"""Parity with the FP64 oracle for the pass plans of the large sizes.

From n = 23 (complex64) the mixer takes two strided high groups per layer, and
their boundaries fuse across layers (layer l's group, layer l + 1's phase and
butterflies in one pass); n = 30, the precision-study size, runs a group of 9
bits with rows of 16 amplitudes and one of 8 bits with rows of 32.  These tests
compare the CUDA path element by element with the oracle's amplitudes at
n = 23..28, for every arithmetic (complex64, complex128, complex128 in
double-float, the halved state), and at n = 30, p = 10 with the oracle's stored
results for five seeded instances (``tests/golden/n30_p10_oracle.json``, written
by ``tests/golden/make_n30_golden.py``, which calls only the oracle).

Tolerances (from the arithmetic; an amplitude passes n p butterfly stages and p
phase products):
  * complex128: amplitudes within 2e-15 (1 + n p) max|psi|, p_succ within 1e-10
    relative, norm within 1e-12;
  * complex64: amplitudes within 1e-6 (1 + n p) max|psi|, p_succ within 1e-4
    relative, norm within 1e-6;
  * complex128 in double-float arithmetic: amplitudes within 2e-12 (1 + n p)
    max|psi|, p_succ within 1e-10 relative;
  * p_succ and norm of a given state (standalone reduction): complex64 within
    8 u = 4.8e-7 relative (each |v|^2 rounded at most 3 times, pairwise FP32
    sums of 32 terms, FP64 above), complex128 within 1e-12.
"""
import functools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api  # noqa: E402
from paper_2401_02852_gb300._lib import DF64, MIXER_RX2B, Z2_HALF  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "n30_p10_oracle.json")
AMP_TOL = {"c64": 1e-6, "c128": 2e-15, "df64": 2e-12}
PS_TOL = {"c64": 1e-4, "c128": 1e-10, "df64": 1e-10}
NORM_TOL = {"c64": 1e-6, "c128": 1e-12, "df64": 1e-10}


@functools.lru_cache(maxsize=2)
def _case(n, sign, p):
    """A satisfiable NAE-5-SAT instance at r = 8 (rejection on the oracle's
    count), its oracle cost table, and the oracle's state and (p_succ, norm)."""
    inst, n_sol = gen.satisfiable_instance("plans", n, 5, 8.0, p, oracle.count_solutions)
    cost, _, _ = oracle.cost_table(n, inst.var, inst.neg)
    g, b = gen.linear_ramp(p)
    psi = oracle.evolve(n, cost, g, b, sign)
    ps, nm = oracle.success_prob(n, cost, psi)
    return inst, n_sol, cost, g, b, psi, ps, nm


def _flags(sign):
    return 0 if sign == 1 else MIXER_RX2B


def _compare(kind, n, p, got_state, psi, ps, nm, ref_ps, ref_nm):
    assert abs(ps - ref_ps) <= PS_TOL[kind] * ref_ps, (ps, ref_ps)
    assert abs(nm - ref_nm) <= NORM_TOL[kind], nm
    amax = float(np.max(np.abs(psi)))
    err = float(np.max(np.abs(got_state.astype(np.complex128) - psi)))
    assert err <= AMP_TOL[kind] * (1 + n * p) * amax, (err, amax)


def test_plan_shapes_of_the_large_sizes():
    """The plans these tests cover: two high groups from n = 23 (complex64) and
    n = 21 (complex128); at n = 30 a full 9-bit group with rows of 16 and a full
    8-bit group with rows of 32."""
    assert api.plan(22, "c64") == [(0, 13, 13), (13, 9, 4)]
    assert api.plan(23, "c64") == [(0, 13, 13), (13, 8, 5), (15, 2, 5)]
    assert api.plan(26, "c64") == [(0, 13, 13), (13, 8, 5), (18, 5, 5)]
    assert api.plan(28, "c64") == [(0, 13, 13), (13, 8, 5), (20, 7, 5)]
    assert api.plan(30, "c64") == [(0, 13, 13), (13, 9, 4), (22, 8, 5)]
    assert api.plan(24, "c128") == [(0, 12, 12), (12, 8, 4), (16, 4, 4)]
    # p = 3 at n = 26: init on a high group, fused boundaries on both high groups,
    # plain low passes, and a plain reducing last pass
    assert api.pass_schedule(26, 3, "c64") == [(1, 0, 0), (0, 0, 1), (2, 0, 2), (0, 1, 1), (1, 1, 2), (0, 2, 1),
                                               (2, 2, 1)]


@pytest.mark.parametrize("n,p,sign,dtype", [(23, 3, 1, "c64"), (23, 3, 1, "c128"), (24, 3, -1, "c64"),
                                            (24, 3, -1, "c128"), (26, 3, 1, "c64"), (26, 3, 1, "c128"),
                                            (26, 2, -1, "c64"), (28, 2, 1, "c64")])
def test_two_high_groups_match_oracle(n, p, sign, dtype):
    inst, n_sol, _, g, b, psi, ref_ps, ref_nm = _case(n, sign, p)
    cost, gsol, _ = api.cost_table(inst)
    assert gsol == n_sol
    st, ps, nm = api.evolve(n, cost, inst.m, g, b, dtype, flags=_flags(sign))
    _compare(dtype, n, p, st.cpu().numpy(), psi, ps, nm, ref_ps, ref_nm)


@pytest.mark.parametrize("n,p,sign", [(24, 3, -1), (26, 3, 1)])
def test_df64_two_high_groups_match_oracle(n, p, sign):
    inst, _, _, g, b, psi, ref_ps, ref_nm = _case(n, sign, p)
    cost, _, _ = api.cost_table(inst)
    st, ps, nm = api.evolve(n, cost, inst.m, g, b, "c128", flags=DF64 | _flags(sign))
    _compare("df64", n, p, st.cpu().numpy(), psi, ps, nm, ref_ps, ref_nm)


@pytest.mark.parametrize("n,p,sign", [(24, 3, -1), (26, 3, 1)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_halved_state_matches_oracle(n, p, sign, dtype):
    """The stored half x < 2^(n-1) equals the oracle's full state there."""
    inst, _, _, g, b, psi, ref_ps, ref_nm = _case(n, sign, p)
    half, _, _ = api.cost_table_half(inst)
    st, ps, nm = api.evolve(n, half, inst.m, g, b, dtype, flags=Z2_HALF | _flags(sign))
    assert st.numel() == 1 << (n - 1)
    _compare(dtype, n, p, st.cpu().numpy(), psi[: 1 << (n - 1)], ps, nm, ref_ps, ref_nm)


@pytest.mark.parametrize("n", [24, 26])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_standalone_success_prob_grid_stride(n, dtype):
    """qaoa_success_prob on states of 2^24 and 2^26 amplitudes: more chunks of
    8192 amplitudes than blocks, so each block strides over several."""
    inst, _, cost_o, g, b, _, _, _ = _case(n, 1 if n == 26 else -1, 3)
    cost, _, _ = api.cost_table(inst)
    st, _, _ = api.evolve(n, cost, inst.m, g, b, dtype, flags=_flags(1 if n == 26 else -1))
    ps, nm = api.success_prob(n, cost, st)
    ref_ps, ref_nm = oracle.success_prob(n, cost_o, st.cpu().numpy().astype(np.complex128))
    tol = 8 * 2.0 ** -24 if dtype == "c64" else 1e-12
    assert abs(ps - ref_ps) <= tol * ref_ps and abs(nm - ref_nm) <= tol * ref_nm


@pytest.mark.parametrize("n,p,sign,dtype", [(24, 3, 1, "c64"), (24, 3, -1, "c128")])
def test_grad_two_high_groups_matches_oracle(n, p, sign, dtype):
    """Adjoint gradient at n = 24 (backward plan: low 12 bits and two high
    groups) against the oracle's stored-state reverse mode."""
    inst, _ = gen.satisfiable_instance("plans-grad", n, 5, 8.0, 0, oracle.count_solutions)
    cost_o, _, _ = oracle.cost_table(n, inst.var, inst.neg)
    g, b = gen.linear_ramp(p)
    rps, rdg, rdb = oracle.grad(n, cost_o, g, b, sign)
    cost, _, _ = api.cost_table(inst)
    ps, dg, db = api.grad(n, cost, inst.m, g, b, dtype, flags=_flags(sign))
    scale = max(np.max(np.abs(rdg)), np.max(np.abs(rdb)))
    tol = (1e-8 if dtype == "c128" else 1e-6 * (1 + n * p)) * scale
    assert abs(ps - rps) <= PS_TOL[dtype] * rps
    assert np.max(np.abs(dg - rdg)) <= tol and np.max(np.abs(db - rdb)) <= tol


# ---------------------------------------------------------------------------
# n = 30, p = 10: the precision-study workload, five seeded instances


def _golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle results for n = 30 are missing")
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.slow
def test_n30_p10_five_instances_match_oracle():
    doc = _golden()
    n, p = doc["n"], doc["p"]
    assert len(doc["instances"]) == 5
    g, b = gen.linear_ramp(p)
    for rec in doc["instances"]:
        # the instance: rejected attempts are unsatisfiable on the GPU's count too
        for a in range(rec["attempt"]):
            assert api.cost_table(gen.raw_instance(doc["tag"], n, doc["k"], doc["r"], rec["index"], a))[1] == 0
        inst = gen.raw_instance(doc["tag"], n, doc["k"], doc["r"], rec["index"], rec["attempt"])
        assert inst.m == rec["m"]
        cost, n_sol, max_c = api.cost_table(inst)
        assert (n_sol, max_c) == (rec["n_sol"], rec["max_cost"])
        xs = torch.tensor(rec["x"], dtype=torch.int64, device="cuda")
        assert cost[xs].cpu().tolist() == rec["cost_x"]
        want = np.array(rec["psi_re"]) + 1j * np.array(rec["psi_im"])
        for kind in ("c64", "c128", "df64"):
            dtype = "c64" if kind == "c64" else "c128"
            st, ps, nm = api.evolve(n, cost, inst.m, g, b, dtype, flags=DF64 if kind == "df64" else 0)
            assert abs(ps - rec["p_succ"]) <= PS_TOL[kind] * rec["p_succ"], (kind, rec["index"], ps)
            assert abs(nm - rec["norm"]) <= NORM_TOL[kind], (kind, rec["index"], nm)
            amax = float(st.abs().max())
            got = st[xs].cpu().numpy().astype(np.complex128)
            assert np.max(np.abs(got - want)) <= AMP_TOL[kind] * (1 + n * p) * amax, (kind, rec["index"])
            del st
            torch.cuda.empty_cache()
        # the halved state: p_succ, and the amplitudes of the sampled x (or of
        # their complements, which the half stores)
        del cost
        torch.cuda.empty_cache()
        half, _, _ = api.cost_table_half(inst)
        st, ps, nm = api.evolve(n, half, inst.m, g, b, "c64", flags=Z2_HALF)
        assert abs(ps - rec["p_succ"]) <= PS_TOL["c64"] * rec["p_succ"]
        assert abs(nm - rec["norm"]) <= NORM_TOL["c64"]
        top = np.uint64(1 << (n - 1))
        xh = np.array(rec["x"], dtype=np.uint64)
        xh = np.where(xh & top, (~xh) & np.uint64((1 << n) - 1), xh).astype(np.int64)
        got = st[torch.from_numpy(xh).cuda()].cpu().numpy().astype(np.complex128)
        amax = float(st.abs().max())
        assert np.max(np.abs(got - want)) <= AMP_TOL["c64"] * (1 + n * p) * amax
        del st, half
        torch.cuda.empty_cache()
