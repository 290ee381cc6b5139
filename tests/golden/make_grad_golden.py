#!/usr/bin/env python
"""Writes ``grad_n22_p20_oracle.json``: the FP64 oracle's gradient for the first
instances of the adjoint-gradient workload (random NAE-5-SAT, n = 22, m = 176,
r = 8, depth p = 20 with the linear ramp, mixer exp(+i beta sum X_j) of
Appendix A.3).

Only the oracle computes here (``oracle.cost_table`` for the satisfiability
filter, ``oracle.grad``: reverse mode with every forward state stored).  The
instances come from the seeded generator (tag "grad-cfg", the workload's own),
attempt 0, 1, ... per index until the oracle's count finds a solution.  Floats
are written with ``repr`` (exact round trip).  Usage:
    python tests/golden/make_grad_golden.py [--count 2]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2401_02852_gb300 import instances as gen  # noqa: E402

TAG, N, K, R, P = "grad-cfg", 22, 5, 8.0, 20


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2)
    ap.add_argument("--out", default=os.path.join(HERE, "grad_n22_p20_oracle.json"))
    args = ap.parse_args()
    gamma, beta = gen.linear_ramp(P)
    doc = {"what": "FP64 oracle gradient of p_succ, NAE-5-SAT n=22 m=176 (r=8), p=20 linear ramp, "
                   "mixer exp(+i beta sum X_j) (Appendix A.3)",
           "writer": "tests/golden/make_grad_golden.py (calls only oracle/)",
           "tag": TAG, "n": N, "k": K, "r": R, "p": P, "instances": []}
    for index in range(args.count):
        t0 = time.time()
        inst, n_sol = gen.satisfiable_instance(TAG, N, K, R, index, oracle.count_solutions)
        cost, _, _ = oracle.cost_table(N, inst.var, inst.neg)
        ps, dg, db = oracle.grad(N, cost, gamma, beta, 1)
        doc["instances"].append({"index": index, "attempt": int(inst.seed_key[-1]), "n_sol": int(n_sol),
                                 "p_succ": float(ps), "dgamma": [float(x) for x in dg],
                                 "dbeta": [float(x) for x in db], "oracle_seconds": round(time.time() - t0, 1)})
        print(f"index {index}: p_succ {ps!r} ({time.time() - t0:.1f} s)", flush=True)
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
