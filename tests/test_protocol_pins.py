"""Pins of the paper's evaluation protocol inputs and fits (no GPU).

* r_hat_k against the expanded closed form 2^(k-1) ln 2 - (ln 2)/2 - 1/4 and its
  leading-order limit (Sec. "QAOA Procedure", Eq. for r_hat^NAE_k);
* the array clause draw: k distinct variables per clause, uniform variables
  and positions, fair negations (chi-square tests);
* m ~ Poisson(r_hat_k n): its mean and variance;
* the ensemble mean of #sol / 2^n under Poisson m equals
  exp(-2^(1-k) r_hat_k n) (each clause is violated by a uniform x with
  probability 2^(1-k), the computation behind the theorem on excessive
  scaling), counted by the oracle's brute force;
* the fits: a power law and a 2^(c n + d) law recovered from exact data.
"""
import math

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2401_02852_gb300 import instances as gen
from paper_2401_02852_gb300 import protocol


def test_threshold_density_closed_form():
    ln2 = math.log(2.0)
    for k in range(2, 16):
        expanded = 2.0 ** (k - 1) * ln2 - ln2 / 2 - 0.25
        assert gen.threshold_density(k) == pytest.approx(expanded, rel=1e-14, abs=1e-14)
    # leading order 2^(k-1) ln 2 (the o_k(1) and lower terms vanish relative to it)
    assert gen.threshold_density(30) / (2.0 ** 29 * ln2) == pytest.approx(1.0, rel=1e-8)
    assert gen.threshold_density(3) == pytest.approx(2.176015131959808, rel=1e-14)


def test_random_assignment_exponent():
    for k in range(3, 11):
        assert protocol.random_assignment_exponent(k) == pytest.approx(2.0 ** (1 - k) * gen.threshold_density(k))
    # tends to ln 2 (the exponent of one satisfying assignment among 2^n) as k grows
    assert protocol.random_assignment_exponent(20) == pytest.approx(math.log(2.0), rel=1e-4)


def test_array_clause_draw_distribution():
    n, k, m = 9, 4, 30000
    var, neg = gen.draw_clauses_keys(n, k, m, gen.rng_for("pin-keys", n, k))
    assert var.shape == (m, k) and var.dtype == np.int32 and neg.dtype == np.uint8
    assert var.min() >= 0 and var.max() < n
    assert all(len(set(row)) == k for row in var[:2000])
    s = np.sort(var, axis=1)
    assert np.all(np.diff(s, axis=1) > 0)
    # every variable equally likely overall and in each position
    for col in [var.reshape(-1), var[:, 0], var[:, k - 1]]:
        counts = np.bincount(col, minlength=n)
        assert scipy.stats.chisquare(counts).pvalue > 1e-3
    # every k-subset equally likely: C(9, 4) = 126 cells
    codes = (s * (n ** np.arange(k))).sum(axis=1)
    _, counts = np.unique(codes, return_counts=True)
    assert counts.size == math.comb(n, k)
    assert scipy.stats.chisquare(counts).pvalue > 1e-3
    assert abs(neg.mean() - 0.5) < 4 * 0.5 / math.sqrt(neg.size)


def test_protocol_instances_poisson_clause_count():
    n, k, count = 12, 5, 600
    ms = np.array([gen.protocol_instance("pin-poisson", n, k, i).m for i in range(count)])
    lam = gen.threshold_density(k) * n
    assert abs(ms.mean() - lam) < 4 * math.sqrt(lam / count)
    # Poisson: variance = mean (sample variance within a generous band)
    assert 0.75 * lam < ms.var(ddof=1) < 1.3 * lam
    inst = gen.protocol_instance("pin-poisson", n, k, 3)
    again = gen.protocol_instance("pin-poisson", n, k, 3)
    assert np.array_equal(inst.var, again.var) and np.array_equal(inst.neg, again.neg)
    assert inst.k == k and inst.var.shape == (inst.m, k)


def test_ensemble_solution_fraction_matches_the_theorem():
    """E[#sol / 2^n] = E[(1 - 2^(1-k))^m] = exp(-2^(1-k) r n) for m ~ Poisson(r n)."""
    n, k, count = 10, 3, 800
    fr = np.array([oracle.count_solutions(gen.protocol_instance("pin-theorem", n, k, i)) / 2 ** n
                   for i in range(count)])
    want = math.exp(-protocol.random_assignment_exponent(k) * n)
    assert abs(fr.mean() - want) < 4 * fr.std(ddof=1) / math.sqrt(count), (fr.mean(), want)


def test_fits_recover_exact_laws():
    ps = [1, 2, 4, 8, 16, 32]
    a, b = protocol.fit_power_law(ps, [0.7 * p ** -0.25 for p in ps])
    assert a == pytest.approx(0.7) and b == pytest.approx(-0.25)
    ns = list(range(12, 20))
    c, d = protocol.fit_bits(ns, [2.0 ** (0.31 * n - 1.5) for n in ns])
    assert c == pytest.approx(0.31) and d == pytest.approx(-1.5)
    pts = {(p, n): {"inv_mean_psucc": 2.0 ** (0.4 * n / p), "median_running_time": 2.0 ** (0.3 * n / p)}
           for p in ps for n in ns}
    ex = protocol.exponents(9, pts, ps, ns)
    assert ex["by_p"][2]["C_hat_bits"] == pytest.approx(0.2)
    assert ex["by_p"][2]["relative_error"] == pytest.approx(0.25)
    assert ex["power_law_bits"][1] == pytest.approx(-1.0)
    assert ex["paper_power_law"] == protocol.PAPER_POWER_LAW[9]


def test_evaluation_batches_and_first_attempts():
    """The evaluation's batches cover every instance index once per n, in
    order, within the memory budget; the prefetched first attempts are the
    instances the rejection sampler would draw itself."""
    ns = list(range(12, 20))
    b = protocol.eval_batches(ns, 2500, "c64", mem_budget=2 << 30)
    for n in ns:
        mine = [(c0, size) for (nn, c0, size) in b if nn == n]
        covered = [i for c0, size in mine for i in range(c0, c0 + size)]
        assert covered == list(range(2500))
        assert all(size * (1 << n) * 9 <= (2 << 30) or size == 1 for _, size in mine)
    assert [nn for nn, _, _ in b] == sorted(nn for nn, _, _ in b)
    got = protocol.first_attempts("pin-first", 13, 7, 5, start=40)
    for i, inst in enumerate(got):
        want = gen.protocol_instance("pin-first", 13, 7, 40 + i, 0)
        assert np.array_equal(inst.var, want.var) and np.array_equal(inst.neg, want.neg)
