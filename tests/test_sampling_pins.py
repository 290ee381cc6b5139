"""Pins of the oracle's bitstring sampler and running time (Sec. "Running Times").

A draw returns x with probability |psi(x)|^2 (inverse CDF in index order, one
caller-supplied uniform per draw); the running time of an instance is the
number of draws up to the first satisfying one.  The pins are closed forms
(uniform and single-point states), invariants (monotone in u, never an x of
probability zero), a chi-square test of the frequencies, and the geometric law
of the running time: its mean over independent draw sequences is 1 / p_succ.
No GPU is used.
"""
import math

import numpy as np
import scipy.stats

import oracle
from paper_2401_02852_gb300 import instances as gen


def test_uniform_state_draws_floor_of_u_times_size():
    # F(x) = (x + 1) / 2^n exactly in FP64, so x_j = floor(u_j 2^n)
    for n in (1, 5, 12):
        psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
        u = gen.uniforms("pin-uniform", 4000, n)
        xs = oracle.sample(n, psi, u)
        assert np.array_equal(xs, np.floor(u * (1 << n)).astype(np.uint64))


def test_single_point_state_always_draws_that_point():
    n = 9
    for x0 in (0, 1, 137, (1 << n) - 1):
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[x0] = np.exp(0.3j)
        xs = oracle.sample(n, psi, gen.uniforms("pin-point", 500, x0))
        assert np.all(xs == x0)


def test_draws_are_monotone_in_u_and_skip_zero_probability():
    n = 10
    psi = gen.random_state("pin-sparse", n, 0, sparsity=0.7)
    u = np.sort(np.concatenate([gen.uniforms("pin-mono", 3000, 0), [0.0, 1.0 - 2.0 ** -53]]))
    xs = oracle.sample(n, psi, u)
    assert np.all(np.diff(xs.astype(np.int64)) >= 0)
    assert np.all(np.abs(psi[xs.astype(np.int64)]) > 0)
    # u = 0 gives the first x of nonzero probability, u -> 1 the last
    nz = np.flatnonzero(np.abs(psi) > 0)
    assert xs[0] == nz[0] and xs[-1] == nz[-1]


def test_frequencies_match_the_born_rule():
    n, draws = 6, 40000
    psi = gen.random_state("pin-born", n, 1)
    xs = oracle.sample(n, psi, gen.uniforms("pin-born", draws, 1))
    expect = draws * np.abs(psi) ** 2
    counts = np.bincount(xs.astype(np.int64), minlength=1 << n)
    _, pval = scipy.stats.chisquare(counts, expect)
    assert pval > 1e-3


def _sat_instance(n, k, m, tag):
    for idx in range(1000):
        var, neg = gen.draw_clauses(n, k, m, gen.rng_for(tag, n, k, m, idx))
        cost, sol, _ = oracle.cost_table(n, var, neg)
        if sol:
            return cost
    raise RuntimeError("no satisfiable instance")


def test_running_time_extremes():
    n = 8
    cost = _sat_instance(n, 3, 14, "pin-rt")
    sol = np.flatnonzero(cost == 0)
    on_sol = np.zeros(1 << n, dtype=np.complex128)
    on_sol[sol] = 1 / math.sqrt(sol.size)
    assert oracle.running_time(n, cost, on_sol, gen.uniforms("pin-rt", 50, 0)) == 1
    off_sol = np.where(cost == 0, 0, 1).astype(np.complex128)
    off_sol /= np.linalg.norm(off_sol)
    assert oracle.running_time(n, cost, off_sol, gen.uniforms("pin-rt", 500, 1)) == 0


def test_running_time_is_geometric_in_p_succ():
    """Draws are independent with success probability p_succ / norm, so the
    running time is geometric: mean 1 / p, variance (1 - p) / p^2."""
    n, p_layers = 10, 3
    cost = _sat_instance(n, 3, 30, "pin-geo")
    g, b = gen.linear_ramp(p_layers)
    psi = oracle.evolve(n, cost, g, b)
    ps, nm = oracle.success_prob(n, cost, psi)
    p = ps / nm
    runs = 3000
    k = int(40 / p) + 1
    rts = np.array([oracle.running_time(n, cost, psi, gen.uniforms("pin-geo", k, i)) for i in range(runs)])
    assert np.all(rts >= 1)  # k draws are enough (the chance of none is (1 - p)^k < e^-40)
    mean, sd = rts.mean(), math.sqrt((1 - p) / p ** 2)
    assert abs(mean - 1 / p) < 4 * sd / math.sqrt(runs), (mean, 1 / p)
