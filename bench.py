#!/usr/bin/env python
"""Benchmark of the QAOA statevector hot path on one or more GB300s.

Workload (the precision-study configuration): random NAE-5-SAT, n = 30,
m = 240 (r = 8), kept if satisfiable, depth p = 10 with linear-ramp angles,
complex64 state (8.6 GB).  One step = the whole hot path for one instance:
cost table (bit-sliced integer kernel), the p-layer evolution (phase fused into
the first pass of each layer, strided high-qubit passes) and p_succ (FP64
reduction fused into the last pass).  Metric: amplitude-layer updates per
second (2^n p per step), summed over ranks.

Prints ONE JSON line (rank 0).  ``roofline`` is the method's 1-pass floor
(17 B per amplitude-layer for complex64) over the measured step time; the pass
kinds' own bandwidths sit beside it.  ``extra`` carries the other configured
workloads, run after the timed region (rank 0, one GPU): the five n = 30
instances against stored FP64-oracle values, the halved state, complex128 and
double-float complex128, the batched gradient (256 x n = 22, p = 20) against
stored oracle gradients plus 200 Adam steps, the scaling sweep (n = 16..32,
200 instances per n), the 20,000-request serving stream at 200/s and a sweep
of offered rates, each arm of the serving comparison on the same state
layout.  ``--quick`` runs the headline alone.  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
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
NOMINAL_HBM_GBPS = 8000.0  # GB300 HBM3e, nominal (about 8 TB/s); the scored fraction uses the measured copy
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


def step_traffic(n: int, p: int, dtype: str, alg: dict):
    """DRAM bytes of one step (cost table + passes) from the committed per-kind
    ncu figures, provided every kind the step launches has a current figure."""
    total, src = 0, None
    launches = {"cost_table": 1, **alg["launches"]}
    for kind, count in launches.items():
        if not count:
            continue
        per, src = profiled_traffic(kind, n, p, dtype)
        if per is None:
            return None, src
        total += per * count
    return total, src


def load_golden(name: str):
    """Stored FP64-oracle results (tests/golden/, written by scripts that call only the oracle)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", name)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def config2_seeds(n: int, p: int, g, b, count: int = 5) -> dict:
    """The precision study's five seeded instances: p_succ of the complex64,
    complex128 and double-float complex128 evolutions against the stored FP64
    oracle values, and each complex64 evolution's time and bandwidth."""
    import torch

    from paper_2401_02852_gb300 import api
    from paper_2401_02852_gb300 import instances as gen
    from paper_2401_02852_gb300._lib import DF64

    gold = load_golden("n30_p10_oracle.json") or {"instances": []}
    by_index = {r["index"]: r for r in gold["instances"]}
    alg = algorithmic_bytes(n, p, "c64")
    sched = alg["pass_low"] + alg["pass_high"]
    cost = torch.empty(1 << n, dtype=torch.uint8, device="cuda")
    st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    st128 = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    rows = []
    for idx in range(count):
        inst, n_sol = gen.satisfiable_instance("bench-n30", n, K_SAT, R_SAT, idx, lambda x: api.cost_table(x)[1])
        api.cost_table(inst, out=cost, stats=False)
        api.evolve(n, cost, inst.m, g, b, "c64", out=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        _, ps, nm = api.evolve(n, cost, inst.m, g, b, "c64", out=st)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        _, ps128, _ = api.evolve(n, cost, inst.m, g, b, "c128", out=st128)
        _, psdf, _ = api.evolve(n, cost, inst.m, g, b, "c128", flags=DF64, out=st128)
        rec = by_index.get(idx)
        ok = rec is not None and rec["attempt"] == inst.seed_key[-1] and rec["n_sol"] == n_sol
        ref = rec["p_succ"] if ok else None
        rows.append({"index": idx, "attempt": int(inst.seed_key[-1]), "n_sol": n_sol, "p_succ_c64": ps, "norm_c64": nm,
                     "ms_per_evolution_c64": ms, "amp_layer_per_s": (2 ** n) * p / (ms / 1e3),
                     "schedule_GBps": sched / (ms / 1e3) / 1e9,
                     "effective_GBps_at_17B": 17 * (2 ** n) * p / (ms / 1e3) / 1e9,
                     "oracle_p_succ": ref,
                     "c64_rel_err_vs_oracle": abs(ps - ref) / ref if ref else None,
                     "c128_rel_err_vs_oracle": abs(ps128 - ref) / ref if ref else None,
                     "df64_rel_err_vs_oracle": abs(psdf - ref) / ref if ref else None})
    del cost, st, st128
    errs = [r["c64_rel_err_vs_oracle"] for r in rows if r["c64_rel_err_vs_oracle"] is not None]
    return {"instances": rows, "oracle_source": "tests/golden/n30_p10_oracle.json",
            "max_c64_rel_err_vs_oracle": max(errs) if errs else None,
            "max_c128_rel_err_vs_oracle": max((r["c128_rel_err_vs_oracle"] for r in rows
                                               if r["c128_rel_err_vs_oracle"] is not None), default=None),
            "max_df64_rel_err_vs_oracle": max((r["df64_rel_err_vs_oracle"] for r in rows
                                               if r["df64_rel_err_vs_oracle"] is not None), default=None)}


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


SINGLE_CORE_N = 20


def cpu_single_core_sample(p: int, min_seconds: float = 4.0) -> dict | None:
    """The same oracle step on one host core (a child process with
    OMP_NUM_THREADS=1, since the thread count is fixed when the library loads),
    on an n = SINGLE_CORE_N instance, for about `min_seconds`."""
    code = (
        "import json, sys, time\n"
        "sys.path.insert(0, %r)\n"
        "import oracle\n"
        "from paper_2401_02852_gb300 import instances as gen\n"
        "n, p = %d, %d\n"
        "inst, _ = gen.satisfiable_instance('bench-cpu1', n, %d, %r, 0, oracle.count_solutions)\n"
        "g, b = gen.linear_ramp(p)\n"
        "steps, dt = 0, 0.0\n"
        "while dt < %r:\n"
        "    t0 = time.perf_counter()\n"
        "    cost, _, _ = oracle.cost_table(n, inst.var, inst.neg)\n"
        "    oracle.success_prob(n, cost, oracle.evolve(n, cost, g, b))\n"
        "    dt += time.perf_counter() - t0\n"
        "    steps += 1\n"
        "print(json.dumps({'steps': steps, 'seconds': dt, 'm': inst.m}))\n"
    ) % (ROOT, SINGLE_CORE_N, p, K_SAT, R_SAT, min_seconds)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        out = json.loads(res.stdout.strip().splitlines()[-1])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None
    n = SINGLE_CORE_N
    return {"value": (2 ** n) * p * out["steps"] / out["seconds"], "unit": UNIT, "cores": 1,
            "sample": f"{out['steps']} steps of one NAE-5-SAT instance n={n}, m={out['m']}, p={p}, "
                      f"{out['seconds']:.1f} s, OMP_NUM_THREADS=1"}


# ---------------------------------------------------------------------------
def run_reference(args, ws, rank):
    """The oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    if ws > 1 and os.environ.get("OMP_NUM_THREADS") == "1":
        # torchrun sets one OpenMP thread per process; the oracle's only process
        # takes the host's cores (read when the oracle's OpenMP runtime loads)
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
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
        cpu["single_core"] = cpu_single_core_sample(args.p)

    # one GPU per rank; ranks beyond the visible GPUs (a gloo check of the
    # multi-rank path) share them
    local = local % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        # nccl (one GPU per rank); QAOA_DIST_BACKEND=gloo lets several ranks
        # share one GPU, to exercise the multi-rank path where only one GPU is
        # at hand (only host barriers and scalar reductions cross ranks)
        backend = os.environ.get("QAOA_DIST_BACKEND", "nccl")
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
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
    state_dtype = state.dtype
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
    dev = "cuda" if dist is not None and dist.get_backend() == "nccl" else "cpu"
    ms_max = 1000.0 * qdist.max_over_ranks(ms / 1000.0, device=dev)
    value = qdist.job_throughput(float((2 ** n) * p * args.steps), ms / 1000.0, device=dev)

    # Roofline (the scored figure): the method's 1-pass floor, (2 es + 1) bytes per
    # amplitude-layer (17 B complex64, 33 B complex128: the state read and
    # written once and the cost byte read once per layer), times the
    # amplitude-layers of a step, over the measured step time.  Extra passes of
    # the schedule do not raise it.  Beside it, each pass kind's achieved
    # bandwidth on the bytes it really moves (its launches' CUDA-event times).
    kinds = prof.stats
    alg = algorithmic_bytes(n, p, dtype)
    peak, peak_src = measured_peak()
    per_unit = 2 * es + 1
    units = (2 ** n) * p
    step_s = ms_max / args.steps / 1000.0
    achieved = per_unit * units / step_s / 1e9
    passes = {}
    for kind in ("pass_low", "pass_high"):
        if kind in kinds and alg["launches"][kind]:
            per_launch = alg[kind] / alg["launches"][kind]
            avg_ms = kinds[kind][1] / kinds[kind][0]
            gbps = per_launch / (avg_ms / 1000.0) / 1e9
            passes[kind] = {"launches_per_step": alg["launches"][kind], "algorithmic_bytes_per_launch": per_launch,
                            "avg_launch_ms": avg_ms, "achieved_GBps": gbps, "frac": gbps / peak}
    traffic, traffic_src = step_traffic(n, p, dtype, alg)
    dom = max(passes, key=lambda k: kinds[k][1]) if passes else None
    roof = {"kernel": "evolution step: cost table + every pass launch + the p_succ reduction", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_source": traffic_src, "peak_source": peak_src,
            "nominal_peak": NOMINAL_HBM_GBPS, "frac_of_nominal": achieved / NOMINAL_HBM_GBPS, "per_unit_bytes": per_unit,
            "unit_name": "amplitude-layer", "units_per_step": units,
            "achieved_pass_frac": passes[dom]["frac"] if dom else None, "dominant_pass_kind": dom,
            "passes": passes, "schedule_bytes_per_step": alg["pass_low"] + alg["pass_high"]}
    pass_ms = sum(kinds.get(k, (0, 0.0))[1] for k in ("pass_low", "pass_high")) / args.steps

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
        # the units of every rank over the slowest rank's time, as for the headline
        e2e = {"value": qdist.job_throughput(float((2 ** n) * p * args.steps), dt, device=dev), "unit": UNIT,
               "h2d_bytes_per_step": int(inst.var.nbytes + inst.neg.nbytes + 2 * 8 * p),
               "d2h_bytes_per_step": 16}

    extra = {"p_succ": results["p_succ"], "norm": results["norm"], "n_sol": n_sol, "m": inst.m,
             "passes_per_layer": len(plan), "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kinds.items()},
             "pass_ms_per_step": pass_ms}
    if "cost_table" in kinds:
        # The table's work, N m clause tests, against the INT32 lanes of the
        # device at the clock sampled during the timed steps (128 per SM per
        # cycle).  The kernel evaluates 32 assignments per 32-bit operation,
        # counts only the lower half of the table (C(not x) = C(x)) and skips
        # the clauses that cannot be violated within a block's assignments.
        ct_ms = kinds["cost_table"][1] / kinds["cost_table"][0]
        clk_now = clk.summary()
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        lanes = sms * 128 * clk_now["sm_mhz"] * 1e6 if clk_now else None
        extra["cost_table"] = {"ms_per_table": ct_ms, "clause_tests": (2 ** n) * inst.m,
                               "clause_tests_per_s": (2 ** n) * inst.m / (ct_ms / 1000.0),
                               "int32_lane_ops_per_s": lanes, "sms": sms,
                               "sm_mhz": clk_now["sm_mhz"] if clk_now else None,
                               "table_bytes_per_s": (2 ** n) / (ct_ms / 1000.0)}
    legs = []  # (name, function) run after the headline, each guarded

    # The extra workloads run in a single-process run only; with several ranks
    # the line carries the replicated headline alone.
    if ws == 1 and n == N_DEFAULT and p == P_DEFAULT and dtype == "c64" and not args.no_config2:
        def config2():
            return config2_seeds(n, p, g, b)
        legs.append(("config2_five_seeds", config2))
    if args.z2 and ws == 1:
        def z2_leg():
            # the halved state (exact by the global-flip symmetry): same p_succ, half the bytes
            from paper_2401_02852_gb300._lib import Z2_HALF
            half = torch.empty(1 << (n - 1), dtype=torch.uint8, device="cuda")
            st_h = torch.empty(1 << (n - 1), dtype=state_dtype, device="cuda")
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
            return {"ms_per_step": ms_h, "amp_layer_per_s": (2 ** n) * p / (ms_h / 1000.0),
                    "p_succ": hres["p"], "p_succ_rel_diff_vs_full": abs(hres["p"] - results["p_succ"]) /
                    results["p_succ"], "stored_state_GB": (2 ** (n - 1)) * es / 1e9}
        legs.append(("z2_halved", z2_leg))
    if args.compare_c128 and dtype == "c64" and ws == 1:
        def c128_leg():
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
            out = {"c128": {"ms_per_evolution": ms128, "amp_layer_per_s": (2 ** n) * p / (ms128 / 1000.0),
                            "p_succ": ps128, "c64_rel_err_vs_c128": abs(results["p_succ"] - ps128) / ps128,
                            "c64_speedup_over_c128": ms128 / (ms / args.steps)}}
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
            out["c128_df64"] = {"ms_per_evolution": msdf, "amp_layer_per_s": (2 ** n) * p / (msdf / 1000.0),
                                "p_succ": psdf, "p_succ_rel_diff_vs_fp64": abs(psdf - ps128) / ps128,
                                "max_amp_diff_vs_fp64_over_max_amp": amp_err, "speedup_over_fp64": ms128 / msdf}
            del st128, std
            return out
        legs.append(("c128_compare", c128_leg))
    if ws == 1:
        from paper_2401_02852_gb300 import workloads
        if not args.no_grad:
            legs.append(("grad", lambda: workloads.grad_workload(batch=256, n=22, p=20, adam_steps=args.adam_steps,
                                                                 fd_instances=1, reference=load_golden("grad_n22_p20_oracle.json"))))
        if not args.no_sweep:
            legs.append(("sweep", lambda: workloads.sweep_workload(ns=range(16, 33, 2), seeds=args.seeds)))
        if not args.no_batch:
            legs.append(("config1_batch", lambda: workloads.batch_workload(
                reference=load_golden("batch_n12_p5_oracle.json"))))
        if args.serve_requests > 0:
            legs.append(("serving", lambda: workloads.serve_workload(count=args.serve_requests, rate_hz=200.0)))
        if not args.no_rate_sweep:
            legs.append(("serving_rate_sweep", lambda: workloads.serve_rate_sweep(
                rates=(1000.0, 2000.0, 5000.0, 20000.0), count=args.rate_sweep_requests)))
    if legs:
        del state
        torch.cuda.empty_cache()
    for name, fn in legs:
        t0 = time.perf_counter()
        try:
            res = fn()
        except Exception as exc:  # one failing leg must not cost the line
            res = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()
        if name == "c128_compare" and "error" not in res:
            extra.update(res)
        else:
            extra[name] = res
        extra.setdefault("leg_seconds", {})[name] = round(time.perf_counter() - t0, 1)

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
        res = workloads.batch_workload(reference=load_golden("batch_n12_p5_oracle.json"))
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
    ap.add_argument("--serve-requests", type=int, default=20000,
                    help="serving stream (Poisson 200/s) reported beside the headline; 0 skips it")
    ap.add_argument("--rate-sweep-requests", type=int, default=3000, help="requests per offered rate of the sweep")
    ap.add_argument("--no-rate-sweep", action="store_true")
    ap.add_argument("--no-config2", action="store_true", help="skip the five n=30 instances against the oracle")
    ap.add_argument("--no-grad", action="store_true", help="skip the batched-gradient workload")
    ap.add_argument("--no-sweep", action="store_true", help="skip the scaling sweep")
    ap.add_argument("--no-batch", action="store_true", help="skip the 100 x n=12 complex128 batch")
    ap.add_argument("--quick", action="store_true", help="headline only (no extra workloads)")
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
    if args.quick:
        args.no_config2 = args.no_grad = args.no_sweep = args.no_rate_sweep = args.no_batch = True
        args.z2 = args.compare_c128 = False
        args.serve_requests = 0
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != "evolve":
        return run_workload(args)
    return run_native(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
