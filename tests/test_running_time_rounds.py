"""Host logic of the running-time rounds (Sec. "Running Times": an instance's
running time is the number of draws up to and including its first
satisfying one), without a GPU.

``sweep.sample_running_times`` draws in rounds of k = first_k, 4 first_k, ...
for the instances still unresolved, in chunks of at most draw_budget draws
per call, and censors an instance still unresolved once k passes max_draws.
Here the batched kernel is replaced by a fake whose instances have known
running times R_i: a round of k draws after d earlier ones reports R_i - d
when d < R_i <= d + k and 0 otherwise, which is what the kernel reports for a
draw sequence whose first satisfying draw is number R_i.
"""
import numpy as np
import pytest
import torch

from paper_2401_02852_gb300 import instances as gen
from paper_2401_02852_gb300 import sweep


class FakeKernel:
    def __init__(self, R):
        self.R = np.asarray(R, dtype=np.int64)
        self.seen = np.zeros(len(R), dtype=np.int64)
        self.calls = []

    def __call__(self, n, cs, st, u, flags=0):
        ids = cs[:, 0].to(torch.int64).numpy()
        assert st.shape[0] == ids.size and tuple(u.shape)[0] == ids.size
        k = int(u.shape[1])
        assert u.dtype == torch.float64 and float(u.min()) >= 0.0 and float(u.max()) < 1.0
        self.calls.append((ids.copy(), k))
        d = self.seen[ids]
        R = self.R[ids]
        got = np.where((R > d) & (R <= d + k), R - d, 0)
        self.seen[ids] += k
        return got


@pytest.fixture
def cpu_uniforms(monkeypatch):
    real = gen.device_uniforms
    monkeypatch.setattr(sweep.gen, "device_uniforms", lambda tag, shape, index=0: real(tag, shape, index, device="cpu"))


def _batch(B):
    costs = torch.zeros((B, 8), dtype=torch.uint8)
    costs[:, 0] = torch.arange(B, dtype=torch.uint8)  # the fake reads the instance from column 0
    return costs, torch.zeros((B, 8), dtype=torch.complex64)


@pytest.mark.parametrize("draw_budget", [16, 1 << 20])  # chunked calls with gathers, then whole-batch calls
def test_rounds_find_each_first_hit_and_censor(cpu_uniforms, monkeypatch, draw_budget):
    R = [1, 4, 5, 20, 85, 300, 10 ** 9]
    fake = FakeKernel(R)
    monkeypatch.setattr(sweep.api, "running_time_batch", fake)
    costs, states = _batch(len(R))
    rt, draws = sweep.sample_running_times(3, costs, states, 0, "rounds", first_k=4, max_draws=256,
                                           draw_budget=draw_budget)
    # rounds of 4, 16, 64, 256 draws: 340 in all before censoring
    assert rt.tolist() == [1, 4, 5, 20, 85, 300, -1]
    assert draws == 4 + 4 + 20 + 20 + 340 + 340 + 340
    assert fake.seen.tolist() == [4, 4, 20, 20, 340, 340, 340]
    ks = sorted({k for _, k in fake.calls})
    assert ks == [4, 16, 64, 256]
    for ids, k in fake.calls:
        assert ids.size * k <= max(draw_budget, k)  # a chunk stays within the budget (at least one instance)
    # every round draws only for instances still unresolved
    for ids, k in fake.calls:
        before = {4: 0, 16: 4, 64: 20, 256: 84}[k]
        assert all(R[i] > before for i in ids)


def test_instances_resolved_in_the_first_round_take_one_call(cpu_uniforms, monkeypatch):
    fake = FakeKernel([3, 1, 2])
    monkeypatch.setattr(sweep.api, "running_time_batch", fake)
    costs, states = _batch(3)
    rt, draws = sweep.sample_running_times(3, costs, states, 0, "one-round", first_k=4)
    assert rt.tolist() == [3, 1, 2] and draws == 12
    assert len(fake.calls) == 1 and fake.calls[0][0].tolist() == [0, 1, 2]
