#!/usr/bin/env python
"""Writes ``n30_p10_oracle.json``: FP64-oracle results for the precision-study
workload (random NAE-5-SAT, n = 30, m = 240, r = 8, depth p = 10 with the
linear ramp, mixer exp(+i beta sum X_j) of Appendix A.3), five satisfiable
seeded instances.

Only the oracle computes here (``oracle.cost_table``, ``oracle.evolve``,
``oracle.success_prob``); the instances come from the seeded generator
(``instances.raw_instance``), attempt 0, 1, ... per index until the oracle's
brute-force count finds a solution (the rejection sampling of
``instances.satisfiable_instance``).  Per instance it stores the attempt taken,
the solution count and largest cost, p_succ and the norm (Def. of the success
probability), and the oracle's amplitudes psi(x) at sampled x: seeded uniform
draws plus the first solutions in index order.  Floats are written with
``repr`` (exact round trip).

Needs about 20 GB of host memory (complex128 state + uint16 table) and several
minutes per instance on 8 cores.  Usage:
    python tests/golden/make_n30_golden.py [--count 5] [--out tests/golden/n30_p10_oracle.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_02852_gb300 import instances as gen  # noqa: E402

TAG, N, K, R, P = "bench-n30", 30, 5, 8.0, 10
N_RANDOM_X, N_SOLUTION_X = 192, 64


def sample_points(index: int, cost: np.ndarray) -> np.ndarray:
    xs = gen.rng_for("n30-golden-xs", index).integers(0, 1 << N, size=N_RANDOM_X, dtype=np.uint64)
    sols = np.flatnonzero(cost == 0)[:N_SOLUTION_X].astype(np.uint64)
    return np.concatenate([xs, sols])


def one_instance(index: int) -> dict:
    t0 = time.time()
    for attempt in range(1000):
        inst = gen.raw_instance(TAG, N, K, R, index, attempt)
        cost, n_sol, max_c = oracle.cost_table(N, inst.var, inst.neg)
        if n_sol > 0:
            break
        del cost
    else:
        raise RuntimeError(f"no satisfiable attempt for index {index}")
    gamma, beta = gen.linear_ramp(P)
    psi = oracle.evolve(N, cost, gamma, beta, 1)
    p_succ, norm = oracle.success_prob(N, cost, psi)
    xs = sample_points(index, cost)
    amps = psi[xs.astype(np.int64)]
    out = {"index": index, "attempt": attempt, "m": inst.m, "n_sol": int(n_sol), "max_cost": int(max_c),
           "p_succ": float(p_succ), "norm": float(norm), "x": [int(x) for x in xs],
           "cost_x": [int(c) for c in cost[xs.astype(np.int64)]],
           "psi_re": [float(a.real) for a in amps], "psi_im": [float(a.imag) for a in amps],
           "oracle_seconds": round(time.time() - t0, 1)}
    del psi, cost
    return out


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=5)
    ap.add_argument("--out", default=os.path.join(HERE, "n30_p10_oracle.json"))
    args = ap.parse_args()
    doc = {"what": "FP64 oracle results, NAE-5-SAT n=30 m=240 (r=8), p=10 linear ramp "
                   "gamma_l=0.8(l-1/2)/p, beta_l=0.8(1-(l-1/2)/p), mixer exp(+i beta sum X_j) (Appendix A.3)",
           "writer": "tests/golden/make_n30_golden.py (calls only oracle/)",
           "tag": TAG, "n": N, "k": K, "r": R, "p": P, "instances": []}
    for index in range(args.count):
        rec = one_instance(index)
        doc["instances"].append(rec)
        print(f"index {index}: attempt {rec['attempt']} n_sol {rec['n_sol']} p_succ {rec['p_succ']!r} "
              f"({rec['oracle_seconds']} s)", flush=True)
        with open(args.out, "w") as f:
            json.dump(doc, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
