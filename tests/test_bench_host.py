"""Host-side helpers of bench.py (no GPU): the schedule's bytes behind the pass
kinds' bandwidths, the reader of the committed ncu traffic figures, and the
loader of the stored oracle results the bench reports its errors against."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")


def test_schedule_bytes_of_the_headline():
    """n = 30, p = 10, complex64: 10 low and 11 high launches; every pass reads
    and writes the 8-byte state, the passes that apply a phase or reduce also
    read the cost byte, the first only writes."""
    alg = bench.algorithmic_bytes(30, 10, "c64")
    N = 2 ** 30
    assert alg["launches"] == {"pass_low": 10, "pass_high": 11}
    assert alg["pass_low"] == 10 * 16 * N
    # init (9 B) + 9 fused passes (17 B) + the plain reducing last pass (17 B)
    assert alg["pass_high"] == 9 * N + 10 * 17 * N
    # about twice the 1-pass floor (21 launches for 10 layers, the first
    # write-only, most of them without the cost byte)
    assert (alg["pass_low"] + alg["pass_high"]) / N == 339 and 339 / (17 * 10) < 2.0


def test_traffic_reader_is_fresh_or_says_why():
    for kind in ("pass_low", "pass_high", "cost_table"):
        val, src = bench.profiled_traffic(kind, 30, 10, "c64")
        assert (isinstance(val, int) and val > 0 and src.endswith(".txt")) or (val is None and "stale" in src)
    assert bench.profiled_traffic("pass_low", 31, 10, "c64") == (None, None)  # no capture for that workload


def test_stored_oracle_results_load():
    doc = bench.load_golden("n30_p10_oracle.json")
    assert doc["n"] == 30 and doc["p"] == 10 and len(doc["instances"]) == 5
    assert all(0 < r["p_succ"] < 1 and abs(r["norm"] - 1) < 1e-12 for r in doc["instances"])
    grad = bench.load_golden("grad_n22_p20_oracle.json")
    assert grad["n"] == 22 and len(grad["instances"][0]["dgamma"]) == 20
    assert bench.load_golden("missing.json") is None
    batch = bench.load_golden("batch_n12_p5_oracle.json")
    assert batch["n"] == 12 and batch["p"] == 5 and len(batch["instances"]) == 100
    assert all(r["n_sol"] > 0 and len(r["cost_sha256"]) == 64 and abs(r["norm"] - 1) < 1e-12
               for r in batch["instances"])
