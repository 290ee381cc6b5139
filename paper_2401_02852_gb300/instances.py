"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no cost table, no state, no success probability).  The
satisfiability filter takes the solution counter as an argument, so each side
(the CUDA library or the CPU oracle) decides satisfiability with its own code.

Instance recipe (Sec. "Random Problems", Def. of CNF(n, k, r); Sec. "Computational
Phase Transitions" for F_k(n, m)):

* m clauses, fixed to round(r * n) (the paper draws m ~ Poisson(r n); that
  variant is ``poisson_m=True``);
* each clause draws k *distinct* variables uniformly (a uniform k-subset in a
  uniformly random order), clauses independently of each other (duplicates
  across clauses allowed: the clauses are drawn with replacement);
* each literal is negated independently with probability 1/2.

The paper's own evaluation draws CNF(n, k, r_hat_k) with m ~ Poisson(r_hat_k n)
at the threshold estimate r_hat_k (``threshold_density``, ``protocol_instance``);
its clauses come from ``draw_clauses_keys``, the same distribution drawn with
whole-array operations.

Literal j of clause i is the variable ``var[i, j]`` (0-based; variable v is
bit v of the assignment index x) negated when ``neg[i, j] == 1``.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np


@dataclass(frozen=True)
class Instance:
    """One NAE-k-SAT instance: ``var`` int32 [m, k], ``neg`` uint8 [m, k]."""

    n: int
    k: int
    var: np.ndarray
    neg: np.ndarray
    seed_key: tuple = ()

    @property
    def m(self) -> int:
        return int(self.var.shape[0])


def _tag_word(tag: str) -> int:
    return int.from_bytes(hashlib.sha256(tag.encode()).digest()[:4], "little")


def rng_for(tag: str, *key: int) -> np.random.Generator:
    """A PCG64 stream keyed by a text tag and integers (n, index, attempt, ...)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([_tag_word(tag), *map(int, key)])))


def clause_count(n: int, r: float) -> int:
    """m = round(r n): the fixed-m reading of CNF(n, k, r)."""
    return int(round(r * n))


def draw_clauses(n: int, k: int, m: int, rng: np.random.Generator):
    """m clauses of k distinct variables with independent fair negations."""
    if not (1 <= k <= n):
        raise ValueError(f"need 1 <= k <= n, got k={k}, n={n}")
    var = np.empty((m, k), dtype=np.int32)
    neg = np.empty((m, k), dtype=np.uint8)
    for i in range(m):
        var[i] = rng.choice(n, size=k, replace=False)
        neg[i] = rng.integers(0, 2, size=k)
    return var, neg


def draw_clauses_keys(n: int, k: int, m: int, rng: np.random.Generator):
    """m clauses as in ``draw_clauses``, drawn as arrays: the k smallest of n
    iid uniform keys per clause (a uniformly random permutation's first k
    entries: a uniform k-subset in a uniformly random order), then k fair
    negations per clause."""
    if not (1 <= k <= n):
        raise ValueError(f"need 1 <= k <= n, got k={k}, n={n}")
    keys = rng.random((m, n))
    var = np.argsort(keys, axis=1)[:, :k].astype(np.int32)
    neg = rng.integers(0, 2, size=(m, k), dtype=np.uint8)
    return np.ascontiguousarray(var), neg


def threshold_density(k: int) -> float:
    """r_hat_k = (2^(k-1) - 1/2 - 1/(4 ln 2)) ln 2: the asymptotic NAE-k-SAT
    satisfiability threshold without its o_k(1) term (Sec. "QAOA Procedure",
    Eq. for r_hat^NAE_k)."""
    ln2 = math.log(2.0)
    return (2.0 ** (k - 1) - 0.5 - 1.0 / (4.0 * ln2)) * ln2


def protocol_instance(tag: str, n: int, k: int, index: int, attempt: int = 0) -> Instance:
    """Attempt ``attempt`` of instance ``index`` of CNF(n, k, r_hat_k): m ~
    Poisson(r_hat_k n) (Def. of CNF(n, k, r)), clauses from ``draw_clauses_keys``."""
    rng = rng_for(tag, n, k, index, attempt)
    m = int(rng.poisson(threshold_density(k) * n))
    var, neg = draw_clauses_keys(n, k, m, rng)
    return Instance(n=n, k=k, var=var, neg=neg, seed_key=(tag, n, k, index, attempt))


def raw_instance(tag: str, n: int, k: int, r: float, index: int, attempt: int = 0,
                 poisson_m: bool = False) -> Instance:
    """Attempt ``attempt`` of instance ``index``: a fresh, unconditioned draw."""
    rng = rng_for(tag, n, k, int(round(r * 1000)), index, attempt)
    m = int(rng.poisson(r * n)) if poisson_m else clause_count(n, r)
    var, neg = draw_clauses(n, k, m, rng)
    return Instance(n=n, k=k, var=var, neg=neg, seed_key=(tag, n, k, r, index, attempt))


def satisfiable_instance(tag: str, n: int, k: int, r: float, index: int,
                         count_solutions: Callable[[Instance], int],
                         max_attempts: int = 10_000, poisson_m: bool = False) -> tuple[Instance, int]:
    """Rejection sampling: attempts 0, 1, ... until ``count_solutions`` is > 0.

    The instance is drawn without bias towards satisfiability (Sec. "QAOA
    Procedure": generate, then confirm).  Returns the instance and its count.
    """
    for a in range(max_attempts):
        inst = raw_instance(tag, n, k, r, index, a, poisson_m=poisson_m)
        c = int(count_solutions(inst))
        if c > 0:
            return inst, c
    raise RuntimeError(f"no satisfiable instance for {tag} n={n} index={index} in {max_attempts} attempts")


def linear_ramp(p: int, scale: float = 0.8):
    """gamma_l = s (l - 1/2)/p, beta_l = s (1 - (l - 1/2)/p), l = 1..p (float64)."""
    l = np.arange(1, p + 1, dtype=np.float64)
    gamma = scale * (l - 0.5) / p
    beta = scale * (1.0 - (l - 0.5) / p)
    return gamma, beta


def random_state(tag: str, n: int, index: int = 0, sparsity: float = 0.0) -> np.ndarray:
    """A seeded synthetic state: complex128 [2^n], re and im standard normal,
    normalised; with `sparsity` > 0 that fraction of the amplitudes is zero.
    (Random numbers only: an input for tests of the samplers.)"""
    rng = rng_for(tag, n, index)
    z = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    if sparsity > 0:
        z[rng.random(1 << n) < sparsity] = 0
    return z / np.sqrt(np.sum(np.abs(z) ** 2))


def uniforms(tag: str, count: int, index: int = 0) -> np.ndarray:
    """`count` seeded uniforms in [0, 1) (the draws of a sampler)."""
    return rng_for(tag, count, index).random(count)


def device_uniforms(tag: str, shape, index: int = 0, device: str = "cuda"):
    """Seeded uniforms in [0, 1) made on the device (torch Philox generator
    seeded from this module's stream), float64 tensor of `shape`."""
    import torch

    seed = int(rng_for(tag, *(int(d) for d in shape), index).integers(0, 2 ** 62))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.rand(tuple(shape), dtype=torch.float64, device=device, generator=g)


def poisson_arrivals(rate_hz: float, count: int, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = rng_for("arrivals", seed, int(rate_hz * 1000), count)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


@dataclass(frozen=True)
class Request:
    """One serving request: an instance plus its depth and ramp angles."""

    instance: Instance
    p: int
    gamma: np.ndarray
    beta: np.ndarray
    arrival_s: float


def serving_requests(count: int, rate_hz: float = 200.0, k: int = 5, r: float = 8.0,
                     n_range=(14, 26), p_range=(1, 20), seed: int = 0,
                     n_override: Optional[Callable[[int], int]] = None) -> list[Request]:
    """Poisson-arrival stream of NAE-k-SAT requests with uniform n and p.

    Instances are unconditioned draws (satisfiability does not change the
    work); n ~ U{n_range}, p ~ U{p_range}, linear-ramp angles.
    """
    arr = poisson_arrivals(rate_hz, count, seed)
    rng = rng_for("serve-shape", seed, count)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    ps = rng.integers(p_range[0], p_range[1] + 1, size=count)
    out = []
    for i in range(count):
        n = int(ns[i]) if n_override is None else int(n_override(i))
        inst = raw_instance(f"serve-{seed}", n, k, r, i)
        g, b = linear_ramp(int(ps[i]))
        out.append(Request(inst, int(ps[i]), g, b, float(arr[i])))
    return out
