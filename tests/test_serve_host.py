"""Host logic of the serving replay driver, without a GPU: requests are
submitted at their (scaled) arrival times, every ticket is waited for, and the
wall time runs from the first submission to the last completion; the latency
summary's percentiles."""
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2401_02852_gb300 import serve


class FakeServer:
    def __init__(self):
        self.t0 = time.perf_counter()
        self.submitted = []  # (offset s, instance)
        self.waited = []

    def submit(self, inst, gamma, beta):
        self.submitted.append((time.perf_counter() - self.t0, inst))
        return 100 + len(self.submitted)

    def wait(self, ticket, timeout_s):
        self.waited.append(ticket)
        i = ticket - 101
        # request i was submitted at 1 ms + i ms and took (i + 1) ms
        return SimpleNamespace(ticket=ticket, t_submit_ns=(1 + i) * 10 ** 6, t_done_ns=(2 + 2 * i) * 10 ** 6)


def _requests(arrivals):
    return [SimpleNamespace(arrival_s=a, instance=f"inst{i}", gamma=[0.1], beta=[0.2]) for i, a in enumerate(arrivals)]


def test_replay_submits_at_arrival_times_and_waits_for_all():
    arrivals = [0.0, 0.03, 0.06, 0.09]
    fs = FakeServer()
    out, wall = serve.replay(fs, _requests(arrivals), time_scale=1.0)
    offs = [t for t, _ in fs.submitted]
    assert [inst for _, inst in fs.submitted] == ["inst0", "inst1", "inst2", "inst3"]
    for off, a in zip(offs, arrivals):
        assert off >= a - 1e-3  # never early
    assert offs[-1] - offs[0] >= 0.09 - 1e-3
    assert fs.waited == [101, 102, 103, 104] and [r.ticket for r in out] == fs.waited
    # first submission at 1 ms, last completion at 2 + 2 * 3 = 8 ms
    assert wall == pytest.approx(7e-3)


def test_replay_time_scale_compresses_the_schedule():
    fs = FakeServer()
    serve.replay(fs, _requests([0.0, 5.0, 10.0]), time_scale=0.0)
    assert fs.submitted[-1][0] < 0.5  # ten seconds of arrivals replayed at once


def test_latency_summary_percentiles():
    lat = np.arange(1, 101, dtype=np.float64) * 1e-3  # 1 .. 100 ms
    s = serve.latency_summary(lat, wall_s=2.0, count=100)
    assert s["inst_per_s"] == pytest.approx(50.0)
    assert s["p50_ms"] == pytest.approx(50.5)
    assert s["p99_ms"] == pytest.approx(99.01)
    assert s["mean_ms"] == pytest.approx(50.5)
    assert s["count"] == 100 and s["wall_s"] == 2.0
