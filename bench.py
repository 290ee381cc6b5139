#!/usr/bin/env python
"""Benchmark of the QAOA statevector hot path on one or more GB300s.

Workload (the precision-study configuration): random NAE-5-SAT, n = 30,
m = 240 (r = 8), kept if satisfiable, depth p = 10 with linear-ramp angles,
complex64 state (8.6 GB).  One step = the whole hot path for one instance:
cost table (bit-sliced integer kernel), the p-layer evolution (phase fused into
the first pass of each layer, strided high-qubit passes) and p_succ (FP64
reduction fused into the last pass).  Metric: amplitude-layer updates per
second (2^n p per step), summed over ranks.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amp-layer updates/s (NAE-5-SAT n=30, p=10, complex64)"
UNIT = "amp-layer/s"
N_DEFAULT, K_SAT, R_SAT, P_DEFAULT = 30, 5, 8.0, 10
CPU_SAMPLE_N = 26  # bounded oracle sample: steps of one n=26 (m=208) instance of the same depth


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def algorithmic_bytes(n: int, p: int, dtype: str):
    """Minimal HBM bytes each launch of the evolution must move, from the
    library's own launch schedule: every pass reads and writes the state once;
    the first pass of layer 0 only writes it (|+> comes from the phase table);
    a pass that applies a phase (fused or phase-at-load) reads the cost table
    once, and so does the last pass (p_succ needs C).  Returns per-kind byte totals and launch counts."""
    from paper_2401_02852_gb300 import api

    es = 8 if dtype == "c64" else 16
    N = 2 ** n
    seq = api.pass_schedule(n, p, dtype)
    out = {"pass_low": 0, "pass_high": 0, "launches": {"pass_low": 0, "pass_high": 0}}
    for i, (pi, _, mode) in enumerate(seq):
        kind = "pass_low" if pi == 0 else "pass_high"
        if mode == 0:
            b = N * (es + 1)
        else:
            b = N * 2 * es + (N if (mode in (2, 3) or i + 1 == len(seq)) else 0)
        out[kind] += b
        out["launches"][kind] += 1
    return out


def profiled_traffic(kind: str, n: int, p: int, dtype: str):
    """DRAM bytes per launch of `kind` (dram__bytes_read.sum + dram__bytes_write.sum,
    averaged over one step's launches of that kind) from the committed ncu summary
    profiles/traffic_n{n}_p{p}_{dtype}.txt, provided the kernel sources it names
    still hash to the value recorded with the capture; otherwise None."""
    path = os.path.join(ROOT, "profiles", f"traffic_n{n}_p{p}_{dtype}.txt")
    try:
        with open(path) as f:
            lines = f.read().splitlines()
    except OSError:
        return None, None
    for ln in lines:
        parts = ln.split()
        if not parts or parts[0].startswith("#") or parts[0] != kind:
            continue
        fields = dict(x.split("=", 1) for x in parts[2:])
        h = hashlib.sha256()
        for name in fields["sources"].split(","):
            with open(os.path.join(ROOT, "paper_2401_02852_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
        if h.hexdigest()[:16] != fields["sources_sha256"]:
            return None, "stale: the kernel sources changed after the capture"
        return int(parts[1]), os.path.relpath(path, ROOT)
    return None, None


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline_sample(p: int, min_seconds: float = 10.0, max_steps: int = 8):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: whole
    steps (cost table + evolution + p_succ) of one n = CPU_SAMPLE_N instance,
    repeated until about `min_seconds` of CPU work."""
    import oracle
    from paper_2401_02852_gb300 import instances as gen

    n = CPU_SAMPLE_N
    inst, _ = gen.satisfiable_instance("bench-cpu", n, K_SAT, R_SAT, 0, oracle.count_solutions)
    g, b = gen.linear_ramp(p)
    steps, dt = 0, 0.0
    while steps < max_steps and dt < min_seconds:
        t0 = time.perf_counter()
        cost, _, _ = oracle.cost_table(n, inst.var, inst.neg)
        psi = oracle.evolve(n, cost, g, b)
        oracle.success_prob(n, cost, psi)
        dt += time.perf_counter() - t0
        steps += 1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": (2 ** n) * p * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle (OpenMP): {steps} steps of one NAE-5-SAT instance n={n}, m={inst.m}, "
                      f"p={p} (cost table + evolution + p_succ), {dt:.1f} s"}, dt


# ---------------------------------------------------------------------------
def run_reference(args, ws, rank):
    """The oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle
    from paper_2401_02852_gb300 import instances as gen

    n, p = CPU_SAMPLE_N, args.p
    inst, _ = gen.satisfiable_instance("bench-cpu", n, K_SAT, R_SAT, 0, oracle.count_solutions)
    g, b = gen.linear_ramp(p)

    def step():
        cost, _, _ = oracle.cost_table(n, inst.var, inst.neg)
        psi = oracle.evolve(n, cost, g, b)
        return oracle.success_prob(n, cost, psi)[0]

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = (2 ** n) * p * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"NAE-5-SAT n={n} m={inst.m} p={p} (bounded CPU sample of the n=30 workload)",
                      "n": n, "p": p, "k": K_SAT, "r": R_SAT},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"one n={n} instance per step: cost table + evolution + p_succ"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_native(args, ws, rank, local):
    import torch

    from paper_2401_02852_gb300 import api
    from paper_2401_02852_gb300 import instances as gen

    # the oracle baseline runs first, before any GPU work (rank 0, one GPU only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, _ = cpu_baseline_sample(args.p)

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n, p = args.n, args.p
    dtype = args.dtype
    es = 8 if dtype == "c64" else 16

    def gpu_count(inst):
        return api.cost_table(inst)[1]

    inst, n_sol = gen.satisfiable_instance("bench-n30", n, K_SAT, R_SAT, rank, gpu_count)
    g, b = gen.linear_ramp(p)
    cost = torch.empty(1 << n, dtype=torch.uint8, device="cuda")
    state = torch.empty(1 << n, dtype=api.TORCH_DTYPE[api.dtype_code(dtype)], device="cuda")
    plan = api.plan(n, dtype)
    results = {}

    def step():
        api.cost_table(inst, out=cost, stats=False)
        _, ps, nm = api.evolve(n, cost, inst.m, g, b, dtype, out=state)
        results["p_succ"], results["norm"] = ps, nm

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = api.launch_count()
    with ClockSampler(local) as clk, api.Profiler() as prof:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    launches = api.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    from paper_2401_02852_gb300 import dist as qdist  # replicas: only scalars cross ranks
    dev = "cuda" if dist is not None else "cpu"
    ms_max = 1000.0 * qdist.max_over_ranks(ms / 1000.0, device=dev)
    value = qdist.job_throughput(float((2 ** n) * p * args.steps), ms / 1000.0, device=dev)

    # roofline of the dominant kernel from the live per-launch events
    kinds = prof.stats
    dom = max(kinds, key=lambda k: kinds[k][1])
    alg = algorithmic_bytes(n, p, dtype)
    peak, peak_src = measured_peak()
    roof = None
    if dom in ("pass_low", "pass_high"):
        per_launch_bytes = alg[dom] / alg["launches"][dom]
        avg_ms = kinds[dom][1] / kinds[dom][0]
        achieved = per_launch_bytes / (avg_ms / 1000.0) / 1e9
        traffic, traffic_src = profiled_traffic(dom, n, p, dtype)
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms}
    # all pass kernels together, and the 1-pass floor (17 B per amp-layer for complex64)
    pass_ms = sum(kinds.get(k, (0, 0.0))[1] for k in ("pass_low", "pass_high")) / args.steps
    floor_bytes = (2 ** n) * p * (2 * es + 1)
    effective = floor_bytes / (ms_max / args.steps / 1000.0) / 1e9

    # end to end through the public API from host memory
    e2e = None
    if not args.no_e2e:
        work = {"cost": cost, "state": state}
        api.psucc_host(inst, g, b, dtype, work=work)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            api.psucc_host(inst, g, b, dtype, work=work)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": (2 ** n) * p * args.steps / dt * ws, "unit": UNIT,
               "h2d_bytes_per_step": int(inst.var.nbytes + inst.neg.nbytes + 2 * 8 * p),
               "d2h_bytes_per_step": 16}

    extra = {"p_succ": results["p_succ"], "norm": results["norm"], "n_sol": n_sol, "m": inst.m,
             "passes_per_layer": len(plan), "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kinds.items()},
             "pass_ms_per_step": pass_ms, "effective_GBps_at_17B": effective if es == 8 else None}
    if args.z2 and rank == 0:
        # the halved state (exact by the global-flip symmetry): same p_succ, half the bytes
        from paper_2401_02852_gb300._lib import Z2_HALF
        half = torch.empty(1 << (n - 1), dtype=torch.uint8, device="cuda")
        st_h = torch.empty(1 << (n - 1), dtype=state.dtype, device="cuda")
        hres = {}

        def step_h():
            api.cost_table_half(inst, out=half, stats=False)
            _, hres["p"], hres["nm"] = api.evolve(n, half, inst.m, g, b, dtype, flags=Z2_HALF, out=st_h)

        for _ in range(3):
            step_h()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(args.steps):
            step_h()
        a1.record()
        torch.cuda.synchronize()
        ms_h = a0.elapsed_time(a1) / args.steps
        extra["z2_halved"] = {"ms_per_step": ms_h, "amp_layer_per_s": (2 ** n) * p / (ms_h / 1000.0),
                              "p_succ": hres["p"], "p_succ_rel_diff_vs_full": abs(hres["p"] - results["p_succ"]) /
                              results["p_succ"], "stored_state_GB": (2 ** (n - 1)) * es / 1e9}
        del half, st_h

    if args.compare_c128 and dtype == "c64" and rank == 0:
        del state
        torch.cuda.empty_cache()
        st128 = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
        api.evolve(n, cost, inst.m, g, b, "c128", out=st128)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        reps = 2
        for _ in range(reps):
            _, ps128, _ = api.evolve(n, cost, inst.m, g, b, "c128", out=st128)
        z.record()
        torch.cuda.synchronize()
        ms128 = a.elapsed_time(z) / reps
        extra["c128"] = {"ms_per_evolution": ms128, "amp_layer_per_s": (2 ** n) * p / (ms128 / 1000.0),
                         "p_succ": ps128, "c64_rel_err_vs_c128": abs(results["p_succ"] - ps128) / ps128,
                         "c64_speedup_over_c128": ms128 / (ms / args.steps - 0.0)}
        # the same complex128 evolution in double-float arithmetic (QAOA_DF64)
        from paper_2401_02852_gb300._lib import DF64
        std = torch.empty_like(st128)
        api.evolve(n, cost, inst.m, g, b, "c128", flags=DF64, out=std)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            _, psdf, _ = api.evolve(n, cost, inst.m, g, b, "c128", flags=DF64, out=std)
        z.record()
        torch.cuda.synchronize()
        msdf = a.elapsed_time(z) / reps
        amp_err = float((std - st128).abs().max().item() / st128.abs().max().item())
        extra["c128_df64"] = {"ms_per_evolution": msdf, "amp_layer_per_s": (2 ** n) * p / (msdf / 1000.0),
                              "p_succ": psdf, "p_succ_rel_diff_vs_fp64": abs(psdf - ps128) / ps128,
                              "max_amp_diff_vs_fp64_over_max_amp": amp_err, "speedup_over_fp64": ms128 / msdf}
        del st128, std

    if args.serve_requests > 0 and rank == 0 and ws == 1:
        from paper_2401_02852_gb300 import workloads
        torch.cuda.empty_cache()
        extra["serving"] = workloads.serve_workload(count=args.serve_requests, rate_hz=200.0)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32" if dtype == "c64" else "f64",
               "data": "synthetic",
               "config": {"workload": f"NAE-5-SAT n={n} m={inst.m} r=8 p={p} linear ramp, {dtype} state, "
                                      "one satisfiable instance per GPU",
                          "n": n, "m": inst.m, "k": K_SAT, "p": p, "state": dtype,
                          "l2": f"inputs larger than L2 (state {(2 ** n) * es / 1e9:.1f} GB, table {(2 ** n) / 1e9:.2f} GB)",
                          "parallelism": f"replicas x{ws}"},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(), "extra": extra}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_workload(args):
    """The other configured workloads: one JSON line each (not the headline)."""
    import torch

    from paper_2401_02852_gb300 import workloads

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    if args.workload == "serve":
        res = workloads.serve_workload(count=args.requests, rate_hz=args.rate)
    elif args.workload == "grad":
        res = workloads.grad_workload(batch=args.batch, n=args.grad_n, p=args.grad_p, adam_steps=args.adam_steps)
    elif args.workload == "sweep":
        res = workloads.sweep_workload(ns=range(args.sweep_n0, args.sweep_n1 + 1, 2), seeds=args.seeds,
                                       out_dir=args.out_dir)
    elif args.workload == "sample":
        res = workloads.sample_workload(n=args.n)
    elif args.workload == "protocol":
        res = workloads.protocol_workload(ks=tuple(int(k) for k in args.ks.split(",")),
                                          ps=tuple(int(p) for p in args.ps.split(",")),
                                          count=args.count, lr=args.lr)
    else:
        res = workloads.batch_workload()
    res["workload"] = args.workload
    res["wall_seconds"] = time.perf_counter() - t0
    print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--p", type=int, default=P_DEFAULT)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare-c128", dest="compare_c128", action="store_false")
    ap.add_argument("--no-z2", dest="z2", action="store_false", help="skip the halved-state measurement")
    ap.add_argument("--serve-requests", type=int, default=1500,
                    help="short serving run (Poisson 200/s) reported beside the headline; 0 skips it")
    ap.add_argument("--workload", choices=["evolve", "serve", "grad", "sweep", "batch", "sample", "protocol"], default="evolve")
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--grad-n", type=int, default=22)
    ap.add_argument("--grad-p", type=int, default=20)
    ap.add_argument("--adam-steps", type=int, default=200)
    ap.add_argument("--sweep-n0", type=int, default=16)
    ap.add_argument("--sweep-n1", type=int, default=32)
    ap.add_argument("--seeds", type=int, default=200)
    ap.add_argument("--out-dir", default=None)
    ap.add_argument("--ks", default="9", help="protocol: clause widths (comma separated)")
    ap.add_argument("--ps", default="1,2,4,8,16,32", help="protocol: depths (comma separated)")
    ap.add_argument("--count", type=int, default=2500, help="protocol: satisfiable instances per (k, n)")
    ap.add_argument("--lr", type=float, default=1e-2, help="protocol: Adam learning rate of the angle training")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != "evolve":
        return run_workload(args)
    return run_native(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
