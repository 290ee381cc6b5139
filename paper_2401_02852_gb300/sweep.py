"""Scaling sweep: median 1/p_succ versus n and its fitted exponent.

For each n, `seeds` satisfiable CNF(n, k, r) instances (rejection sampling,
satisfiability decided by the bit-exact cost table), each evaluated at every
depth in `ps` with the linear-ramp angles.  Per (n, p) the median of 1/p_succ
is fitted as 2^(c n + d) (Sec. "Running Times": exponents are fitted to a
power law of the form 2^(c n + d), in bits).  With `running_times`, each
instance's running time (bitstrings drawn from its output state until one
satisfies it, Sec. "Running Times") is sampled on the GPU, and the median over
instances is reported beside 1 / E[p_succ].  Results are written one file per
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


def sample_running_times(n: int, costs, states, flags: int, tag: str, first_k: int = 1024,
                         max_draws: int = 1 << 26, draw_budget: int = 1 << 27):
    """Running time of every instance of a batch: rounds of k draws (k growing
    4x per round) for the instances still without a satisfying draw; an
    instance still unresolved after `max_draws` draws is censored (-1).
    Returns the running times and the number of draws taken."""
    B = states.shape[0]
    rt = np.zeros(B, dtype=np.int64)
    done = np.zeros(B, dtype=np.int64)  # draws taken so far
    open_ = np.arange(B)
    k, rnd = first_k, 0
    while open_.size and k <= max_draws:
        step = max(1, draw_budget // k)
        for c0 in range(0, open_.size, step):
            idx = open_[c0:c0 + step]
            u = gen.device_uniforms(tag, (idx.size, k), rnd * 1_000_003 + int(idx[0]))
            if idx.size == B:  # every instance: no gather
                cs, st = costs, states
            else:
                sel = torch.as_tensor(idx, device=states.device)
                cs, st = costs.index_select(0, sel), states.index_select(0, sel)
            got = api.running_time_batch(n, cs, st, u, flags=flags)
            hit = got > 0
            rt[idx[hit]] = done[idx[hit]] + got[hit]
            done[idx] += k
        open_ = open_[rt[open_] == 0]
        k *= 4
        rnd += 1
    rt[open_] = -1
    return rt, int(done.sum())


def run_sweep(ns=range(16, 33, 2), ps=(1, 4, 10, 20), seeds: int = 200, k: int = 5, r: float = 8.0,
              dtype: str = "c64", out_dir: Optional[str] = None, mem_budget: int = 48 << 30, log=print,
              running_times: bool = False):
    es = 8 if dtype == "c64" else 16
    results = {}
    amp_layers = 0
    t_gpu = 0.0
    t_rt = 0.0
    draws = 0
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
        rts = {p: [] for p in todo}
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
                if running_times:
                    t1 = time.perf_counter()
                    rt_b, nd = sample_running_times(n, costs, states, api.Z2_HALF, f"rt-n{n}-p{p}-c{c0}")
                    rts[p].extend(int(x) for x in rt_b)
                    draws += nd
                    t_rt += time.perf_counter() - t1
            del states, costs
            torch.cuda.empty_cache()
        for p in todo:
            arr = np.array(psucc[p])
            rec = {"n": n, "p": p, "k": k, "r": r, "seeds": seeds, "median_inv_psucc": float(np.median(1.0 / arr)),
                   "mean_psucc": float(arr.mean()), "mean_nsol_frac": float(np.mean(nsol) / 2 ** n),
                   "psucc": psucc[p]}
            if running_times:
                rt = np.array(rts[p])
                # censored instances (-1) count as longer than any observed time
                rt_med = np.median(np.where(rt < 0, np.iinfo(np.int64).max, rt))
                rec.update({"median_running_time": float(rt_med), "inv_mean_psucc": float(1.0 / arr.mean()),
                            "censored_running_times": int(np.sum(rt < 0)), "running_times": rts[p]})
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
            rpts = sorted((n, results[(n, p)]["median_running_time"]) for n in ns
                          if (n, p) in results and "median_running_time" in results[(n, p)])
            if len(rpts) >= 2:
                cr, dr = fit_exponent([a for a, _ in rpts], [v for _, v in rpts])
                fits[p].update({"running_time_c_bits": cr, "running_time_d": dr, "running_time_points": rpts})
    return {"results": results, "fits": fits, "random_assignment_bits": random_assignment_exponent_bits(k, r),
            "amp_layer_per_s": amp_layers / t_gpu if t_gpu else None, "gpu_seconds": t_gpu,
            "running_time_seconds": t_rt, "draws": draws}
