"""The native serving loop: results are the same alone and in a mix, match the
oracle, and the host-side controls (cancel, timeouts, budget) behave."""
import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300._lib import QaoaError  # noqa: E402
from paper_2401_02852_gb300.serve import Server, replay  # noqa: E402


def _req(n, p, idx, tag="srv"):
    inst = gen.raw_instance(tag, n, 5, 8.0, idx)
    g, b = gen.linear_ramp(p)
    return inst, g, b


def test_results_same_alone_and_in_mix():
    probes = [_req(12, 5, 0), _req(14, 7, 1), _req(17, 4, 2), _req(20, 3, 3)]
    with Server("c64", n_streams=3) as s:
        alone = [s.wait(s.submit(*r)) for r in probes]
        rng = gen.rng_for("mix", 0)
        others = [_req(int(rng.integers(12, 21)), int(rng.integers(1, 9)), 100 + i) for i in range(40)]
        tickets = []
        for i, o in enumerate(others):
            tickets.append(s.submit(*o))
            if i % 10 == 5:
                tickets.append(("probe", s.submit(*probes[(i // 10) % len(probes)]), (i // 10) % len(probes)))
        mixed = {}
        for t in tickets:
            if isinstance(t, tuple):
                mixed.setdefault(t[2], []).append(s.wait(t[1]))
            else:
                assert s.wait(t).status == 0
        st = s.stats()
    assert st["packed_launches"] >= 1 and st["single_launches"] >= 1
    for j, results in mixed.items():
        for r in results:
            assert r.p_succ == alone[j].p_succ and r.norm == alone[j].norm, (j, r, alone[j])
            assert r.n_sol == alone[j].n_sol


@pytest.mark.parametrize("z2", [False, True])
def test_results_same_alone_and_batched(z2):
    """Requests of one shape (n, m, p, angles) that wait together run as one
    batched pass sequence; each result equals the request's result alone, bit
    for bit, and the batched runs match the oracle."""
    from paper_2401_02852_gb300._lib import Z2_HALF
    flags = Z2_HALF if z2 else 0
    same = [_req(17, 5, 200 + i, tag="grp") for i in range(6)] + [_req(20, 3, 300 + i, tag="grp") for i in range(3)]
    with Server("c64", n_streams=1, flags=flags) as s:
        alone = [s.wait(s.submit(*r)) for r in same]
        assert s.stats()["grouped_requests"] == 0
        blocker = s.submit(*_req(24, 20, 0, tag="grp-block"))  # holds the only slot while the others queue
        tickets = [s.submit(*r) for r in same]
        assert s.wait(blocker, 300).status == 0
        grouped = [s.wait(t, 300) for t in tickets]
        st = s.stats()
    assert st["grouped_requests"] >= 6, st
    for a, b in zip(alone, grouped):
        assert b.status == 0 and (b.p_succ, b.norm, b.n_sol, b.max_cost) == (a.p_succ, a.norm, a.n_sol, a.max_cost)
    for (inst, g, b), r in zip(same[:2] + same[6:7], grouped[:2] + grouped[6:7]):
        cost, sol, _ = oracle.cost_table(inst.n, inst.var, inst.neg)
        ref_ps, _ = oracle.success_prob(inst.n, cost, oracle.evolve(inst.n, cost, g, b))
        assert r.n_sol == sol
        assert abs(r.p_succ - ref_ps) <= 1e-4 * ref_ps + 1e-300


@pytest.mark.parametrize("n,p", [(10, 3), (14, 6), (16, 4), (19, 2)])
def test_serving_matches_oracle(n, p):
    inst, g, b = _req(n, p, 7, tag="srv-orc")
    cost, sol, mx = oracle.cost_table(n, inst.var, inst.neg)
    ref_ps, ref_nm = oracle.success_prob(n, cost, oracle.evolve(n, cost, g, b))
    with Server("c64") as s:
        r = s.wait(s.submit(inst, g, b))
    assert r.status == 0 and r.n_sol == sol and r.max_cost == mx
    if sol:
        assert abs(r.p_succ - ref_ps) <= 1e-4 * ref_ps
    assert abs(r.norm - 1) < 1e-6


def test_replay_and_counters():
    reqs = gen.serving_requests(60, rate_hz=2000.0, n_range=(12, 18), p_range=(1, 6), seed=3)
    with Server("c64", n_streams=2) as s:
        res, wall = replay(s, reqs)
        st = s.stats()
        it = s.issue_time()
    assert st["submitted"] == st["completed"] == 60 and st["errors"] == 0
    launches = st["packed_launches"] + st["single_launches"] + (1 if st["grouped_requests"] else 0)
    assert it["issues"] >= launches and 0 < it["issue_s"] < it["span_s"]
    assert all(r.status == 0 and r.t_submit_ns <= r.t_start_ns <= r.t_done_ns for r in res)
    assert wall > 0


def test_cancel_and_timeout():
    with Server("c64", n_streams=1) as s:
        big = [s.submit(*_req(24, 20, i, tag="slow")) for i in range(3)]
        t = s.submit(*_req(12, 2, 9))
        assert s.cancel(t) or True  # cancelled if still waiting, else it runs to completion
        r = s.wait(t, 120)
        assert r.status in (0, -6)
        with pytest.raises(QaoaError):
            s.wait(big[-1], 1e-6)  # deadline passes before a 20-layer n=24 request finishes
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(QaoaError):
                s.wait(big[-1], bad)
        for b in big:
            assert s.wait(b, 300).status == 0
        with pytest.raises(QaoaError):
            s.poll(big[0])  # retired tickets are unknown


def test_budget_limits_resident_bytes():
    budget = 3 * (1 << 22) * 9  # three n=22 complex64 requests (table + state)
    with Server("c64", hbm_budget_bytes=budget, n_streams=6) as s:
        ts = [s.submit(*_req(22, 2, i, tag="bud")) for i in range(8)]
        assert all(s.wait(t, 300).status == 0 for t in ts)
        st = s.stats()
    assert st["peak_bytes"] <= budget
    with Server("c64", hbm_budget_bytes=1 << 20) as s:
        with pytest.raises(QaoaError):
            s.submit(*_req(22, 2, 0, tag="bud"))  # larger than the whole budget


def test_invalid_request_rejected_at_submit():
    inst = gen.Instance(n=5, k=2, var=np.array([[1, 1]], np.int32), neg=np.zeros((1, 2), np.uint8))
    with Server("c64") as s:
        with pytest.raises(QaoaError):
            s.submit(inst, [0.1], [0.2])
        with pytest.raises(QaoaError):
            s.submit(*_req(12, 1, 0)[:1], [float("nan")], [0.1])
        assert s.stats()["submitted"] == 0


def test_halved_state_server_matches_full():
    """With QAOA_Z2_HALF the unpacked requests run on the halved state: same
    p_succ (complex64 tolerance), same solution counts, half the footprint."""
    from paper_2401_02852_gb300._lib import Z2_HALF
    reqs = [_req(n, p, 30 + n, tag="srv-z2") for n, p in ((15, 3), (18, 5), (21, 2), (24, 4))]
    with Server("c64") as s:
        full = [s.wait(s.submit(*r)) for r in reqs]
    with Server("c64", flags=Z2_HALF) as s:
        half = [s.wait(s.submit(*r)) for r in reqs]
        peak = s.stats()["peak_bytes"]
    for a, b in zip(full, half):
        assert b.status == 0 and a.n_sol == b.n_sol and a.max_cost == b.max_cost
        assert abs(a.p_succ - b.p_succ) <= 1e-5 * a.p_succ and abs(b.norm - 1) < 1e-6
    assert peak <= (1 << 23) * 9  # the largest request's half table + half state
