#!/usr/bin/env python
"""Writes ``batch_n12_p5_oracle.json``: FP64-oracle results for the batched
small-instance workload (random NAE-3-SAT, n = 12, m = 24 (r = 2), depth p = 5
with the linear ramp, mixer exp(+i beta sum X_j) of Appendix A.3), 100
satisfiable seeded instances, the ones the batched benchmark evolves in one
launch.

Only the oracle computes here (``oracle.cost_table``, ``oracle.evolve``,
``oracle.success_prob``); the instances come from the seeded generator
(``instances.raw_instance``), attempt 0, 1, ... per index until the oracle's
brute-force count finds a solution (the rejection sampling of
``instances.satisfiable_instance``).  Per instance it stores the attempt taken,
the solution count and largest cost, the SHA-256 of the whole uint8 cost table
(C(x) <= m = 24 fits a byte), p_succ and the norm (Def. of the success
probability), and the oracle's amplitudes at 16 seeded x.  Floats are written
with ``repr`` (exact round trip).  A few seconds on one core.  Usage:
    python tests/golden/make_batch_golden.py [--out tests/golden/batch_n12_p5_oracle.json]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_02852_gb300 import instances as gen  # noqa: E402

TAG, N, K, R, P, COUNT, N_X = "batch-cfg", 12, 3, 2.0, 5, 100, 16


def one_instance(index: int) -> dict:
    for attempt in range(1000):
        inst = gen.raw_instance(TAG, N, K, R, index, attempt)
        cost, n_sol, max_c = oracle.cost_table(N, inst.var, inst.neg)
        if n_sol > 0:
            break
    else:
        raise RuntimeError(f"no satisfiable attempt for index {index}")
    gamma, beta = gen.linear_ramp(P)
    psi = oracle.evolve(N, cost, gamma, beta, 1)
    p_succ, norm = oracle.success_prob(N, cost, psi)
    xs = gen.rng_for("batch-golden-xs", index).integers(0, 1 << N, size=N_X)
    table = np.ascontiguousarray(cost.astype(np.uint8))
    return {"index": index, "attempt": attempt, "m": inst.m, "n_sol": int(n_sol), "max_cost": int(max_c),
            "cost_sha256": hashlib.sha256(table.tobytes()).hexdigest(),
            "p_succ": float(p_succ), "norm": float(norm), "x": [int(x) for x in xs],
            "psi_re": [float(psi[x].real) for x in xs], "psi_im": [float(psi[x].imag) for x in xs]}


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "batch_n12_p5_oracle.json"))
    args = ap.parse_args()
    doc = {"what": "FP64 oracle results, NAE-3-SAT n=12 m=24 (r=2), p=5 linear ramp "
                   "gamma_l=0.8(l-1/2)/p, beta_l=0.8(1-(l-1/2)/p), mixer exp(+i beta sum X_j) (Appendix A.3)",
           "writer": "tests/golden/make_batch_golden.py (calls only oracle/)",
           "tag": TAG, "n": N, "k": K, "r": R, "p": P,
           "instances": [one_instance(i) for i in range(COUNT)]}
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"wrote {len(doc['instances'])} instances to {args.out}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
