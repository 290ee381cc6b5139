"""The stored oracle results under ``tests/golden/`` still describe the
instances the seeded generator draws today (no GPU).  The GPU tests and the
benchmark compare against these files where the oracle cannot run in their
time; if the generator's streams or the oracle changed, they would silently
compare different instances.  Each check is cheap: the small batch file is
recomputed outright on a few instances, the large files are pinned through
the clause counts at their stored points and the solution counts."""
import hashlib
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_02852_gb300 import instances as gen  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("index", [0, 37, 99])
def test_batch_file_recomputes(index):
    """n = 12, p = 5: the same attempt is the first satisfiable one, the cost
    table hashes to the stored digest, and the oracle gives the stored p_succ,
    norm and amplitudes (within 1e-13)."""
    doc = _load("batch_n12_p5_oracle.json")
    rec = doc["instances"][index]
    n, k, r, p = doc["n"], doc["k"], doc["r"], doc["p"]
    for a in range(rec["attempt"]):  # the earlier attempts are unsatisfiable
        inst = gen.raw_instance(doc["tag"], n, k, r, index, a)
        assert oracle.count_solutions(inst) == 0
    inst = gen.raw_instance(doc["tag"], n, k, r, index, rec["attempt"])
    cost, n_sol, max_c = oracle.cost_table(n, inst.var, inst.neg)
    assert (n_sol, max_c, inst.m) == (rec["n_sol"], rec["max_cost"], rec["m"])
    assert hashlib.sha256(np.ascontiguousarray(cost.astype(np.uint8)).tobytes()).hexdigest() == rec["cost_sha256"]
    g, b = gen.linear_ramp(p)
    psi = oracle.evolve(n, cost, g, b, 1)
    ps, nm = oracle.success_prob(n, cost, psi)
    # the same FP64 arithmetic; 1e-13 leaves room for another libm's last bit
    assert ps == pytest.approx(rec["p_succ"], rel=1e-13) and nm == pytest.approx(rec["norm"], rel=1e-13)
    xs = np.array(rec["x"])
    amp = np.abs(psi).max()
    assert np.allclose(psi[xs].real, rec["psi_re"], rtol=0, atol=1e-13 * amp)
    assert np.allclose(psi[xs].imag, rec["psi_im"], rtol=0, atol=1e-13 * amp)


def test_n30_file_matches_the_generator():
    """n = 30: every stored point's clause count is what the oracle counts for
    the regenerated instance, one x at a time, and the stored solutions are
    solutions."""
    doc = _load("n30_p10_oracle.json")
    for rec in doc["instances"]:
        inst = gen.raw_instance(doc["tag"], doc["n"], doc["k"], doc["r"], rec["index"], rec["attempt"])
        assert inst.m == rec["m"]
        xs = np.array(rec["x"], dtype=np.uint64)
        assert np.array_equal(oracle.cost_samples(inst.var, inst.neg, xs), np.array(rec["cost_x"]))
        assert 0 < rec["n_sol"] and rec["cost_x"].count(0) >= 1


def test_grad_file_matches_the_generator():
    """n = 22: the stored attempt is the first satisfiable one and its
    solution count is the oracle's."""
    doc = _load("grad_n22_p20_oracle.json")
    for rec in doc["instances"]:
        for a in range(rec["attempt"] + 1):
            inst = gen.raw_instance(doc["tag"], doc["n"], doc["k"], doc["r"], rec["index"], a)
            c = oracle.count_solutions(inst)
            assert (c == 0) if a < rec["attempt"] else (c == rec["n_sol"])
