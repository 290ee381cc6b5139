"""Scaling sweep: median 1/p_succ versus n and its fitted exponent.

For each n, `seeds` satisfiable CNF(n, k, r) instances (rejection sampling,
satisfiability decided by the bit-exact cost table), each evaluated at every
depth in `ps` with the linear-ramp angles.  Per (n, p) the median of 1/p_succ
is fitted as 2^(c n + d) (Sec. "Running Times": exponents are fitted to a
power law of the form 2^(c n + d), in bits).  Results are written one file per
(n, p) and skipped when present, so an interrupted sweep resumes.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Iterable, Optional

import numpy as np
import torch

from . import api
from . import instances as gen


def random_assignment_exponent_bits(k: int, r: float) -> float:
    """log2(1/p_succ) per variable when the state stays |+> (gamma = 0 or beta = 0,
    Appendix B) for fixed m = r n: p_succ = (1 - 2^(1-k))^m on average."""
    return -r * math.log2(1.0 - 2.0 ** (1 - k))


def fit_exponent(ns: Iterable[int], values: Iterable[float]):
    """Least squares of log2(values) = c n + d; returns (c, d)."""
    ns = np.asarray(list(ns), dtype=np.float64)
    y = np.log2(np.asarray(list(values), dtype=np.float64))
    A = np.stack([ns, np.ones_like(ns)], axis=1)
    (c, d), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(c), float(d)


def run_sweep(ns=range(16, 33, 2), ps=(1, 4, 10, 20), seeds: int = 200, k: int = 5, r: float = 8.0,
              dtype: str = "c64", out_dir: Optional[str] = None, mem_budget: int = 48 << 30, log=print):
    es = 8 if dtype == "c64" else 16
    results = {}
    amp_layers = 0
    t_gpu = 0.0
    for n in ns:
        todo = [p for p in ps if not (out_dir and os.path.exists(os.path.join(out_dir, f"n{n}_p{p}.json")))]
        for p in ps:
            if p not in todo:
                with open(os.path.join(out_dir, f"n{n}_p{p}.json")) as f:
                    results[(n, p)] = json.load(f)
        if not todo:
            continue
        # The halved state (exact: NAE's global-flip symmetry) halves memory and bytes.
        per = (1 << (n - 1)) * (1 + es)
        chunk = int(max(1, min(seeds, mem_budget // per)))
        psucc = {p: [] for p in todo}
        nsol = []
        for c0 in range(0, seeds, chunk):
            B = min(chunk, seeds - c0)
            costs = torch.empty((B, 1 << (n - 1)), dtype=torch.uint8, device="cuda")
            insts = []
            for j in range(B):
                def count(inst, j=j):
                    return api.cost_table_half(inst, out=costs[j])[1]
                inst, s = gen.satisfiable_instance(f"sweep-k{k}", n, k, r, c0 + j, count)
                insts.append(inst)
                nsol.append(s)
            m = insts[0].m
            states = torch.empty((B, 1 << (n - 1)), dtype=api.TORCH_DTYPE[api.dtype_code(dtype)], device="cuda")
            for p in todo:
                g, b = gen.linear_ramp(p)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, ps_b, _ = api.evolve_batch(n, costs, m, g, b, dtype, flags=api.Z2_HALF, out=states)
                t_gpu += time.perf_counter() - t0
                amp_layers += B * (1 << n) * p
                psucc[p].extend(float(x) for x in ps_b)
            del states, costs
            torch.cuda.empty_cache()
        for p in todo:
            arr = np.array(psucc[p])
            rec = {"n": n, "p": p, "k": k, "r": r, "seeds": seeds, "median_inv_psucc": float(np.median(1.0 / arr)),
                   "mean_psucc": float(arr.mean()), "mean_nsol_frac": float(np.mean(nsol) / 2 ** n),
                   "psucc": psucc[p]}
            results[(n, p)] = rec
            if out_dir:
                os.makedirs(out_dir, exist_ok=True)
                with open(os.path.join(out_dir, f"n{n}_p{p}.json"), "w") as f:
                    json.dump(rec, f)
            if log:
                log(f"n={n} p={p}: median 1/p_succ = {rec['median_inv_psucc']:.4g}")
    fits = {}
    for p in ps:
        pts = sorted((n, results[(n, p)]["median_inv_psucc"]) for n in ns if (n, p) in results)
        if len(pts) >= 2:
            c, d = fit_exponent([a for a, _ in pts], [v for _, v in pts])
            fits[p] = {"c_bits": c, "d": d, "points": pts}
    return {"results": results, "fits": fits, "random_assignment_bits": random_assignment_exponent_bits(k, r),
            "amp_layer_per_s": amp_layers / t_gpu if t_gpu else None, "gpu_seconds": t_gpu}
