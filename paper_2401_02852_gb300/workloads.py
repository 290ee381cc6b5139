"""Benchmark workloads beyond the headline evolution (driven by ``bench.py``).

* ``serve``:  a Poisson stream of NAE-5-SAT requests (n ~ U{14..26},
  p ~ U{1..20}, r = 8, linear ramps) through the native serving loop, against
  one request per launch on the same GPU and the same state layout;
  ``serve_rate_sweep`` repeats it at offered rates up to saturation;
* ``grad``:   batched adjoint gradients (256 instances, n = 22, p = 20) checked
  against central differences and, when given, stored FP64 oracle gradients,
  then Adam on the shared angles;
* ``sweep``:  median 1/p_succ versus n and its fitted exponent, and the median
  running time (bitstrings sampled until one satisfies) beside 1/E[p_succ];
* ``batch``:  100 small instances (n = 12, p = 5, complex128) in one launch;
* ``sample``: bitstring draws from the n = 30, p = 10 output state, and
  running times of a batch of protocol-sized states (n = 19);
* ``protocol``: the paper's own evaluation (``protocol``): angles trained at
  n = 12 per (k, p), then p_hat and median running times over satisfiable
  CNF(n, k, r_hat_k) instances at n = 12..19, and the fitted exponents.

Every function returns a JSON-serialisable dict.  All device work goes through
the library's C ABI.
"""
from __future__ import annotations

import time
from typing import Optional

import numpy as np
import torch

from . import api, protocol, serve, sweep, train
from . import instances as gen


def _sync():
    torch.cuda.synchronize()


def _serve_arms(reqs, warm, n_streams: int, z2: bool, baseline: bool) -> dict:
    """One request stream through the native server and, optionally, one
    request per launch on the same GPU, both on the same state layout."""
    flags = api.Z2_HALF if z2 else 0
    with serve.Server("c64", n_streams=n_streams, flags=flags) as s:
        for rq in warm:
            s.wait(s.submit(rq.instance, rq.gamma, rq.beta))
        res, wall = serve.replay(s, reqs)
        stats = s.stats()
        issue = s.issue_time()
    lat = np.array([r.latency_s for r in res])
    count = len(reqs)
    amp_layers = sum((1 << rq.instance.n) * rq.p for rq in reqs)
    out = {"server": serve.latency_summary(lat, wall, count) | {"amp_layer_per_s": amp_layers / wall},
           "server_stats": stats, "server_issue": issue, "errors": int(sum(r.status != 0 for r in res))}
    if baseline:
        work = {}
        for rq in warm:
            api.psucc_host(rq.instance, rq.gamma, rq.beta, "c64", work=work)
        base_ps, base_lat, base_wall = serve.one_per_launch(reqs, flags=flags)
        out["one_per_launch"] = serve.latency_summary(base_lat, base_wall, count)
        ps = np.array([r.p_succ for r in res])
        bp = np.array(base_ps)
        mask = bp > 0
        out["max_rel_diff_vs_one_per_launch"] = (float(np.max(np.abs(ps[mask] - bp[mask]) / bp[mask]))
                                                 if mask.any() else 0.0)
        out["speedup_inst_per_s"] = out["server"]["inst_per_s"] / out["one_per_launch"]["inst_per_s"]
        out["p99_ratio"] = out["one_per_launch"]["p99_ms"] / out["server"]["p99_ms"]
    return out


def serve_workload(count: int = 20000, rate_hz: float = 200.0, n_range=(14, 26), p_range=(1, 20),
                   n_streams: int = 4, seed: int = 0, baseline: bool = True, z2: bool = False) -> dict:
    """The configured serving stream (Poisson arrivals).  Both arms use the same
    state layout: the full state, or with ``z2`` the halved state for every
    request above the packing limit (n > 14) in both."""
    reqs = gen.serving_requests(count, rate_hz=rate_hz, n_range=n_range, p_range=p_range, seed=seed)
    warm = gen.serving_requests(16, rate_hz=1e6, n_range=n_range, p_range=p_range, seed=seed + 1)
    out = {"requests": count, "rate_hz": rate_hz, "n_range": list(n_range), "p_range": list(p_range),
           "state_layout": "halved (both arms)" if z2 else "full (both arms)"}
    out.update(_serve_arms(reqs, warm, n_streams, z2, baseline))
    return out


def serve_rate_sweep(rates=(200.0, 1000.0, 2000.0, 5000.0, 20000.0), count: int = 3000, n_range=(14, 26),
                     p_range=(1, 20), n_streams: int = 4, z2: bool = False) -> dict:
    """Offered rates from light load to past saturation (the same request mix at
    each rate, its own seeded stream): instances/s, p50 and p99 of the server
    and of one request per launch."""
    warm = gen.serving_requests(16, rate_hz=1e6, n_range=n_range, p_range=p_range, seed=99)
    rows = []
    for i, rate in enumerate(rates):
        reqs = gen.serving_requests(count, rate_hz=rate, n_range=n_range, p_range=p_range, seed=100 + i)
        r = _serve_arms(reqs, warm, n_streams, z2, True)
        rows.append({"offered_per_s": rate, "requests": count,
                     "server": {k: r["server"][k] for k in ("inst_per_s", "p50_ms", "p99_ms")},
                     "one_per_launch": {k: r["one_per_launch"][k] for k in ("inst_per_s", "p50_ms", "p99_ms")},
                     "speedup_inst_per_s": r["speedup_inst_per_s"],
                     "grouped_requests": r["server_stats"]["grouped_requests"],
                     "packed_launches": r["server_stats"]["packed_launches"],
                     "single_launches": r["server_stats"]["single_launches"],
                     "server_issue_share": r["server_issue"]["issue_share"],
                     "server_mean_issue_us": r["server_issue"]["mean_issue_us"],
                     "max_rel_diff_vs_one_per_launch": r["max_rel_diff_vs_one_per_launch"], "errors": r["errors"]})
    return {"state_layout": "halved (both arms)" if z2 else "full (both arms)", "n_range": list(n_range),
            "p_range": list(p_range), "rates": rows}


def grad_workload(batch: int = 256, n: int = 22, p: int = 20, adam_steps: int = 200, lr: float = 0.01,
                  fd_instances: int = 2, seed_tag: str = "grad-cfg", checkpoint=None,
                  reference: Optional[dict] = None) -> dict:
    """Batched adjoint gradients; ``reference`` (optional) holds stored FP64
    results for the first instances ({"instances": [{"index", "attempt",
    "p_succ", "dgamma", "dbeta"}, ...]}) that the complex64 and complex128
    gradients are compared with."""
    m = gen.clause_count(n, 8.0)
    insts = []
    for i in range(batch):
        inst, _ = gen.satisfiable_instance(seed_tag, n, 5, 8.0, i, lambda x: api.cost_table(x)[1])
        insts.append(inst)
    costs, _, _ = api.cost_table_batch(insts)
    g0, b0 = gen.linear_ramp(p)
    work = (torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda"),
            torch.empty((batch, 1 << n), dtype=torch.complex64, device="cuda"))
    api.grad_batch(n, costs, m, g0, b0, "c64", work=work)  # warm-up
    _sync()
    with api.Profiler() as prof:
        t0 = time.perf_counter()
        ps, dg, db = api.grad_batch(n, costs, m, g0, b0, "c64", work=work)
        _sync()
        t_grad = time.perf_counter() - t0
    # per-kind roofline: algorithmic bytes of each launch kind over its event time
    es, N = 8, batch * (1 << n)
    kinds = prof.stats
    roof = {}
    for kind, (count, ms) in kinds.items():
        if kind in ("adjoint_low", "adjoint_high"):
            per = 4 * es * N + (N if kind == "adjoint_low" else 0)  # psi and lam read + written (+ C)
        elif kind in ("pass_low", "pass_high"):
            per = None  # forward passes: counted from the schedule below
        else:
            continue
        if per:
            roof[kind] = {"launches": count, "ms": ms, "GBps": per * count / (ms * 1e-3) / 1e9}
    fwd_bytes = 0
    seq = api.pass_schedule(n, p, "c64")
    for i, (pi, _, mode) in enumerate(seq):
        last = i + 1 == len(seq)
        fwd_bytes += N * (es + 1) if mode == 0 else N * 2 * es + (N if mode in (2, 3) or last else 0)
        if last:
            fwd_bytes += N * es  # the adjoint seed lam_p = P psi_p written beside the state
    fwd_ms = sum(kinds.get(k, (0, 0.0))[1] for k in ("pass_low", "pass_high"))
    roof["forward"] = {"launches": len(seq), "ms": fwd_ms, "GBps": fwd_bytes / (fwd_ms * 1e-3) / 1e9}
    # central differences (h = 1e-4) on the complex128 evolution of a few instances
    fd = []
    h = 1e-4
    for i in range(fd_instances):
        c = costs[i].contiguous()
        ps128, dg128, db128 = api.grad(n, c, m, g0, b0, "c128")
        f = lambda gg, bb: api.evolve(n, c, m, gg, bb, "c128")[1]
        err_g, err_b, scale = 0.0, 0.0, max(np.max(np.abs(dg128)), np.max(np.abs(db128)))
        for l in range(p):
            e = np.zeros(p)
            e[l] = h
            fdg = (f(g0 + e, b0) - f(g0 - e, b0)) / (2 * h)
            fdb = (f(g0, b0 + e) - f(g0, b0 - e)) / (2 * h)
            err_g = max(err_g, abs(fdg - dg128[l]))
            err_b = max(err_b, abs(fdb - db128[l]))
        fd.append({"instance": i, "c128_vs_fd_max_abs_over_max_grad": max(err_g, err_b) / scale,
                   "c64_vs_c128_max_abs_over_max_grad": float(max(np.max(np.abs(dg[i] - dg128)),
                                                                  np.max(np.abs(db[i] - db128))) / scale),
                   "c64_psucc_rel_err_vs_c128": abs(ps[i] - ps128) / ps128})
    vs_ref = []
    for rec in (reference or {}).get("instances", []):
        i = int(rec["index"])
        if i >= batch or insts[i].seed_key[-1] != rec["attempt"]:
            continue
        rdg, rdb = np.array(rec["dgamma"]), np.array(rec["dbeta"])
        scale = max(np.max(np.abs(rdg)), np.max(np.abs(rdb)))
        ps128, dg128, db128 = api.grad(n, costs[i].contiguous(), m, g0, b0, "c128")
        vs_ref.append({"instance": i,
                       "c64_grad_max_abs_err_over_max_grad": float(max(np.max(np.abs(dg[i] - rdg)),
                                                                       np.max(np.abs(db[i] - rdb))) / scale),
                       "c128_grad_max_abs_err_over_max_grad": float(max(np.max(np.abs(dg128 - rdg)),
                                                                        np.max(np.abs(db128 - rdb))) / scale),
                       "c64_psucc_rel_err": abs(float(ps[i]) - rec["p_succ"]) / rec["p_succ"],
                       "c128_psucc_rel_err": abs(ps128 - rec["p_succ"]) / rec["p_succ"]})
    del work
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    if adam_steps > 0:
        g1, b1, trace = train.train_angles(costs, n, m, g0, b0, steps=adam_steps, lr=lr, checkpoint=checkpoint)
    else:
        g1, b1, trace = g0, b0, [(0, float(np.mean(np.log(np.maximum(ps, 1e-300)))))]
    _sync()
    t_adam = time.perf_counter() - t0
    # one gradient = forward (p layers) + reverse sweep (p layers on two states)
    amp_layers = batch * (1 << n) * p
    peak = None
    try:
        import json as _json
        import os as _os
        with open(_os.path.join(_os.path.dirname(_os.path.dirname(_os.path.abspath(__file__))),
                                "MEASURED_PEAKS.json")) as f:
            peak = float(_json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass
    if peak:
        for v in roof.values():
            v["frac_of_measured_peak"] = v["GBps"] / peak
    return {"batch": batch, "n": n, "m": m, "p": p, "grad_seconds": t_grad, "roofline_by_kind": roof,
            "grad_amp_layer_per_s_forward_equiv": amp_layers / t_grad, "mean_psucc_initial": float(np.mean(ps)),
            "fd_checks": fd, "vs_oracle": vs_ref, "adam_steps": adam_steps, "adam_seconds": t_adam,
            "objective_first": trace[0][1], "objective_last": trace[-1][1],
            "trace_every_20": [t for t in trace if t[0] % 20 == 0 or t[0] == len(trace) - 1],
            "gamma_final": list(map(float, g1)), "beta_final": list(map(float, b1))}


def sweep_workload(ns=range(16, 33, 2), ps=(1, 4, 10, 20), seeds: int = 200, out_dir=None,
                   running_times: bool = True) -> dict:
    res = sweep.run_sweep(ns=ns, ps=ps, seeds=seeds, out_dir=out_dir, log=None, running_times=running_times)
    table = {f"n{n}_p{p}": r["median_inv_psucc"] for (n, p), r in sorted(res["results"].items())}
    out = {"seeds": seeds, "ns": list(ns), "ps": list(ps), "median_inv_psucc": table,
           "fits_bits": {str(p): {"c": f["c_bits"], "d": f["d"]} for p, f in res["fits"].items()},
           "random_assignment_bits": res["random_assignment_bits"],
           "amp_layer_per_s": res["amp_layer_per_s"], "gpu_seconds": res["gpu_seconds"]}
    if running_times:
        out["median_running_time"] = {f"n{n}_p{p}": r.get("median_running_time")
                                      for (n, p), r in sorted(res["results"].items())}
        out["inv_mean_psucc"] = {f"n{n}_p{p}": r.get("inv_mean_psucc") for (n, p), r in sorted(res["results"].items())}
        out["censored_running_times"] = sum(r.get("censored_running_times", 0) for r in res["results"].values())
        out["running_time_fits_bits"] = {str(p): {"c": f.get("running_time_c_bits"), "d": f.get("running_time_d")}
                                         for p, f in res["fits"].items()}
        out["running_time_seconds"] = res["running_time_seconds"]
        out["draws"] = res["draws"]
        out["draws_per_s"] = res["draws"] / res["running_time_seconds"] if res["running_time_seconds"] else None
    return out


def batch_workload(count: int = 100, n: int = 12, k: int = 3, r: float = 2.0, p: int = 5, reps: int = 20,
                   reference: Optional[dict] = None) -> dict:
    """One launch evolving ``count`` small instances (complex128, FP64 and
    double-float).  ``reference`` (optional) holds stored FP64 results of the
    same instances ({"instances": [{"index", "attempt", "n_sol", "cost_sha256",
    "p_succ"}, ...]}): the cost tables are compared byte for byte (by hash) and
    p_succ relatively."""
    insts = [gen.satisfiable_instance("batch-cfg", n, k, r, i, lambda x: api.cost_table(x)[1])[0]
             for i in range(count)]
    costs, sols, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(p)
    states = torch.empty((count, 1 << n), dtype=torch.complex128, device="cuda")
    api.evolve_batch(n, costs, insts[0].m, g, b, "c128", out=states)
    _sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        _, ps, nm = api.evolve_batch(n, costs, insts[0].m, g, b, "c128", out=states)
    _sync()
    dt = (time.perf_counter() - t0) / reps
    # FP64 work of the whole-evolution kernel: per amplitude and layer, n factored
    # butterfly stages (one FMA per component: 2 FMA per amplitude each) and the
    # phase multiply (4 FMA-equivalents); 2 flops per FMA.
    flops = count * (1 << n) * p * (2 * n + 4) * 2
    fp64_nominal = 1.25e12  # GB300 dense FP64, nominal (not measured here)
    # the same batch in double-float arithmetic (QAOA_DF64)
    from ._lib import DF64
    stdf = torch.empty_like(states)
    api.evolve_batch(n, costs, insts[0].m, g, b, "c128", flags=DF64, out=stdf)
    _sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        _, psdf, _ = api.evolve_batch(n, costs, insts[0].m, g, b, "c128", flags=DF64, out=stdf)
    _sync()
    dtdf = (time.perf_counter() - t0) / reps
    sol = sols > 0
    vs_ref = None
    if reference is not None:
        import hashlib

        recs = {rec["index"]: rec for rec in reference["instances"]}
        tables = costs.cpu().numpy()
        same_inst = same_table = 0
        rel, rel_df = [], []
        for i, inst in enumerate(insts):
            rec = recs.get(i)
            if rec is None or rec["attempt"] != inst.seed_key[-1]:
                continue
            same_inst += 1
            h = hashlib.sha256(np.ascontiguousarray(tables[i]).tobytes()).hexdigest()
            same_table += int(h == rec["cost_sha256"] and int(sols[i]) == rec["n_sol"])
            rel.append(abs(ps[i] - rec["p_succ"]) / rec["p_succ"])
            rel_df.append(abs(psdf[i] - rec["p_succ"]) / rec["p_succ"])
        vs_ref = {"instances": same_inst, "cost_tables_bit_exact": same_table,
                  "max_c128_rel_err": float(max(rel)) if rel else None,
                  "max_df64_rel_err": float(max(rel_df)) if rel_df else None}
    return {"count": count, "n": n, "m": insts[0].m, "p": p, "ms_per_batch": dt * 1e3,
            "amp_layer_per_s": count * (1 << n) * p / dt,
            "roofline": {"bound": "fp64", "achieved_tflops": flops / dt / 1e12, "peak_tflops": fp64_nominal / 1e12,
                         "frac": flops / dt / fp64_nominal, "peak_source": "nominal"},
            "mean_psucc": float(np.mean(ps)),
            "max_norm_err": float(np.max(np.abs(nm - 1))), "mean_nsol": float(np.mean(sols)),
            "df64": {"ms_per_batch": dtdf * 1e3, "speedup_over_fp64": dt / dtdf,
                     "max_psucc_rel_diff_vs_fp64": float(np.max(np.abs(psdf[sol] - ps[sol]) / ps[sol])),
                     "max_amp_diff_vs_fp64": float((stdf - states).abs().max())},
            "vs_oracle": vs_ref}


def protocol_workload(ks=(9,), ps=(1, 2, 4, 8, 16, 32), count: int = 2500, lr: float = 1e-2) -> dict:
    res = protocol.run_protocol(ks=ks, ps=ps, count=count, lr=lr)
    evolve_s = sum(v["stats"]["evolve_s"] for v in res["by_k"].values())
    amp_layers = sum(v["stats"]["amp_layers"] for v in res["by_k"].values())
    draws = sum(v["stats"]["draws"] for v in res["by_k"].values())
    sample_s = sum(v["stats"]["sample_s"] for v in res["by_k"].values())
    res["evolve_amp_layer_per_s"] = amp_layers / evolve_s if evolve_s else None
    res["draws_per_s"] = draws / sample_s if sample_s else None
    return res


def _event_ms(fn, reps: int) -> float:
    """Mean device time of `fn` over `reps` calls on the current stream (CUDA events)."""
    fn()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def sample_workload(n: int = 30, p: int = 10, draws: int = 1 << 24, batch: int = 2500, batch_n: int = 19,
                    batch_k: int = 9, batch_p: int = 8, batch_draws: int = 4096, reps: int = 5) -> dict:
    """Draw throughput of the sampler.  (a) One n = 30 state (the headline
    evolution): the two-level prefix alone (one draw) and with `draws` draws.
    (b) Running times of `batch` evolved CNF(batch_n, batch_k, r_hat) states,
    `batch_draws` uniforms each, as the protocol's first sampling round."""
    inst, _ = gen.satisfiable_instance("bench-n30", n, 5, 8.0, 0, lambda x: api.cost_table(x)[1])
    cost = api.cost_table(inst)[0]
    g, b = gen.linear_ramp(p)
    state, _, _ = api.evolve(n, cost, inst.m, g, b, "c64")
    u1 = gen.device_uniforms("sample-bench", (1,))
    u = gen.device_uniforms("sample-bench", (draws,))
    out = torch.empty(draws, dtype=torch.int64, device="cuda")
    t_scan = _event_ms(lambda: api.sample(n, state, u1, out=out[:1]), reps)
    t_all = _event_ms(lambda: api.sample(n, state, u, out=out), reps)
    N = 1 << n
    res = {"single": {"n": n, "p": p, "draws": draws, "prefix_ms": t_scan, "ms": t_all,
                      "draws_per_s": draws / ((t_all - t_scan) * 1e-3),
                      "prefix_GBps": N * 8 / (t_scan * 1e-3) / 1e9,
                      "prefix_fp64_gflops": 3 * N / (t_scan * 1e-3) / 1e9}}
    del state, cost, u, out
    torch.cuda.empty_cache()
    insts = [gen.protocol_instance("sample-bench", batch_n, batch_k, i) for i in range(batch)]
    costs, _, _ = api.cost_table_batch(insts)
    g, b = gen.linear_ramp(batch_p)
    states, _, _ = api.evolve_batch(batch_n, costs, max(i.m for i in insts), g, b, "c64")
    ub = gen.device_uniforms("sample-bench-batch", (batch, batch_draws))
    rts = {}

    def run():
        rts["rt"] = api.running_time_batch(batch_n, costs, states, ub)

    t_b = _event_ms(run, reps)
    res["batch"] = {"n": batch_n, "k": batch_k, "p": batch_p, "instances": batch, "draws_each": batch_draws,
                    "ms": t_b, "draws_per_s": batch * batch_draws / (t_b * 1e-3),
                    "resolved": int(np.sum(rts["rt"] > 0))}
    return res
