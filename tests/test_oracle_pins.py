"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
tables, closed forms, dense matrix exponentials, the random-assignment theorem,
exact counting identities and symmetries.  No GPU is used.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2401_02852_gb300 import instances as gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inst(tag, n, k, m, idx=0):
    rng = gen.rng_for(tag, n, k, m, idx)
    return gen.draw_clauses(n, k, m, rng)


def _sat_inst(tag, n, k, m):
    """First satisfiable draw of the tag's stream (so p_succ is not identically 0)."""
    for idx in range(1000):
        var, neg = _inst(tag, n, k, m, idx)
        cost, sol, _ = oracle.cost_table(n, var, neg)
        if sol:
            return var, neg, cost
    raise RuntimeError("no satisfiable instance")


# --------------------------------------------------------------------------
# Cost table C(x)


def test_hand_derived_tables():
    """Tables enumerated by hand from the NAE definition (Sec. 'Problem Hamiltonian')."""
    with open(os.path.join(GOLDEN, "hand_cost_tables.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        cost, sol, mx = oracle.cost_table(c["n"], np.array(c["var"]), np.array(c["neg"]))
        assert cost.tolist() == c["cost"], c["name"]
        assert sol == c["n_sol"], c["name"]
        assert mx == max(c["cost"])


@pytest.mark.parametrize("n,k,m", [(5, 2, 7), (8, 3, 16), (10, 5, 40), (12, 7, 30), (9, 9, 5), (6, 1, 4)])
def test_clause_count_identity(n, k, m):
    """Each clause on k distinct variables is violated by exactly 2 * 2^(n-k) of the
    2^n assignments (the all-false and all-true settings of its k literals; the
    per-clause probability 2^(1-k) of Appendix B), so sum_x C(x) = m 2^(n-k+1)."""
    var, neg = _inst("identity", n, k, m)
    cost, _, _ = oracle.cost_table(n, var, neg)
    assert int(cost.astype(np.int64).sum()) == m * 2 ** (n - k + 1)


@pytest.mark.parametrize("n,k,m", [(7, 3, 14), (11, 5, 60), (13, 4, 40)])
def test_global_flip_symmetry(n, k, m):
    """C(x) = C(not x): the Z2 symmetry of NAE-SAT under a global bit flip (Sec. 2.2)."""
    var, neg = _inst("flip", n, k, m)
    cost, _, _ = oracle.cost_table(n, var, neg)
    x = np.arange(1 << n)
    assert np.array_equal(cost, cost[(~x) & ((1 << n) - 1)])


@pytest.mark.parametrize("n,k,m", [(6, 3, 12), (10, 5, 50), (9, 2, 20)])
def test_nae_as_sat_lemma(n, k, m):
    """Appendix A.4's lemma: x satisfies a clause under NAE iff both x and its
    complement satisfy it as an ordinary disjunction.  Counted here with that
    formulation (an 'any literal true' test on x and on not-x), independent of
    the oracle's 'all literals equal' test."""
    var, neg = _inst("lemma", n, k, m)
    cost, sol, _ = oracle.cost_table(n, var, neg)
    x = np.arange(1 << n, dtype=np.int64)
    ref = np.zeros(1 << n, dtype=np.int64)
    for i in range(m):
        lits = np.stack([((x >> int(var[i, j])) & 1) ^ int(neg[i, j]) for j in range(k)])
        sat_x = lits.any(axis=0)
        sat_flip = (1 - lits).any(axis=0)
        ref += ~(sat_x & sat_flip)
    assert np.array_equal(cost.astype(np.int64), ref)
    assert sol == int((ref == 0).sum())


def test_cost_samples_match_table():
    n, k, m = 12, 5, 96
    var, neg = _inst("samples", n, k, m)
    cost, _, _ = oracle.cost_table(n, var, neg)
    xs = gen.rng_for("xs", 1).integers(0, 1 << n, size=500).astype(np.uint64)
    assert np.array_equal(oracle.cost_samples(var, neg, xs), cost[xs.astype(np.int64)])


def test_solution_density_matches_theorem():
    """Appendix B: for an unconditioned random instance with m clauses,
    E[#sol / 2^n] = (1 - 2^(1-k))^m exactly (clauses independent, each violated
    by a fixed x with probability 2^(1-k)).  Statistical check over 400 draws."""
    n, k, m = 10, 3, 10
    vals = []
    for idx in range(400):
        var, neg = _inst("density", n, k, m, idx)
        _, sol, _ = oracle.cost_table(n, var, neg)
        vals.append(sol / 2 ** n)
    vals = np.array(vals)
    expect = (1 - 2.0 ** (1 - k)) ** m
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(vals.mean() - expect) < 4 * se + 1e-12


def test_invalid_inputs_rejected():
    with pytest.raises(ValueError):
        oracle.cost_table(3, np.array([[0, 1, 3]]), np.array([[0, 0, 0]]))  # variable out of range


# --------------------------------------------------------------------------
# State evolution


def _closed_form_n1(gamma, beta, sign):
    """n = 1, C = [0, 1] (one 'clause' violated at x = 1), one layer:
    psi_0 = (cos b + i s sin b e^{-i g}) / sqrt 2, so
    p(0) = (1 + s sin(2b) sin(g)) / 2."""
    return 0.5 * (1.0 + sign * math.sin(2 * beta) * math.sin(gamma))


@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("g,b", [(0.3, 0.2), (1.1, -0.7), (-2.0, 0.45), (0.0, 1.3)])
def test_n1_closed_form(sign, g, b):
    cost = np.array([0, 1], dtype=np.uint16)
    psi = oracle.evolve(1, cost, [g], [b], sign)
    ps, norm = oracle.success_prob(1, cost, psi)
    assert abs(ps - _closed_form_n1(g, b, sign)) < 1e-15
    assert abs(norm - 1) < 1e-15


def _dense_state(n, cost, gamma, beta, sign):
    """prod_i expm(i s beta_i B) expm(-i gamma_i diag C) |+>, B = sum_j X_j,
    qubit j acting on bit j of the index (dense 2^n x 2^n matrices)."""
    N = 1 << n
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    B = np.zeros((N, N), dtype=complex)
    for j in range(n):
        # kron order: most significant bit first, so bit j sits at position n-1-j
        op = np.array([[1]], dtype=complex)
        for q in reversed(range(n)):
            op = np.kron(op, X if q == j else np.eye(2))
        B += op
    psi = np.full(N, 2 ** (-n / 2), dtype=complex)
    for g, b in zip(gamma, beta):
        psi = np.exp(-1j * g * cost.astype(float)) * psi
        psi = scipy.linalg.expm(1j * sign * b * B) @ psi
    return psi


@pytest.mark.parametrize("n,k,m,p", [(3, 3, 4, 1), (5, 3, 10, 3), (8, 4, 20, 2), (6, 2, 9, 4)])
@pytest.mark.parametrize("sign", [1, -1])
def test_dense_matrix_exponential(n, k, m, p, sign):
    var, neg, cost = _sat_inst("dense", n, k, m)
    rng = gen.rng_for("dense-angles", n, p)
    gamma, beta = rng.uniform(-1.5, 1.5, p), rng.uniform(-1.5, 1.5, p)
    psi = oracle.evolve(n, cost, gamma, beta, sign)
    ref = _dense_state(n, cost, gamma, beta, sign)
    assert np.max(np.abs(psi - ref)) < 1e-12


@pytest.mark.parametrize("sign", [1, -1])
def test_p1_brute_force(sign):
    """One layer: psi(x) = 2^{-n/2} sum_y cos^{n-d}(b) (i s sin b)^d e^{-i g C(y)},
    d = Hamming(x, y), from expanding prod_j [cos b I + i s sin b X_j]."""
    n, k, m = 7, 3, 12
    var, neg, cost = _sat_inst("p1", n, k, m)
    g, b = 0.61, 0.37
    psi = oracle.evolve(n, cost, [g], [b], sign)
    N = 1 << n
    y = np.arange(N)
    ph = np.exp(-1j * g * cost.astype(float))
    ref = np.empty(N, dtype=complex)
    for x in range(N):
        d = np.array([bin(x ^ int(t)).count("1") for t in y])
        ref[x] = 2 ** (-n / 2) * np.sum(np.cos(b) ** (n - d) * (1j * sign * np.sin(b)) ** d * ph)
    assert np.max(np.abs(psi - ref)) < 1e-13


def _fwht(a):
    a = a.copy()
    h = 1
    while h < a.shape[0]:
        a = a.reshape(-1, 2, h)
        a = np.stack([a[:, 0] + a[:, 1], a[:, 0] - a[:, 1]], axis=1).reshape(-1)
        h *= 2
    return a


@pytest.mark.parametrize("n", [4, 9, 12])
def test_mixer_via_walsh_hadamard(n):
    """exp(i s b sum_j X_j) = H^n diag(exp(i s b (n - 2|y|))) H^n (a textbook
    identity: X = H Z H).  A second mixer built on the fast Walsh-Hadamard
    transform, checked against the oracle's butterflies over several layers."""
    k, m, p, sign = 3, 2 * n, 3, 1
    var, neg, cost = _sat_inst("fwht", n, k, m)
    gamma, beta = gen.linear_ramp(p)
    N = 1 << n
    weight = np.array([bin(t).count("1") for t in range(N)])
    psi = np.full(N, 2 ** (-n / 2), dtype=complex)
    for g, b in zip(gamma, beta):
        psi = psi * np.exp(-1j * g * cost.astype(float))
        psi = _fwht(np.exp(1j * sign * b * (n - 2 * weight)) * _fwht(psi)) / N
    assert np.max(np.abs(oracle.evolve(n, cost, gamma, beta, sign) - psi)) < 1e-12


@pytest.mark.parametrize("which", ["p0", "gamma0", "beta0"])
def test_random_assignment_theorem(which):
    """Appendix B: with gamma = 0 or beta = 0 every layer only multiplies |+> by a
    global phase, so p_succ = #sol / 2^n (and trivially so at p = 0)."""
    n, k, m = 10, 3, 20
    for idx in range(20):
        var, neg = _inst("thm", n, k, m, idx)
        cost, sol, _ = oracle.cost_table(n, var, neg)
        if sol:
            break
    p = 0 if which == "p0" else 4
    g, b = gen.linear_ramp(p)
    if which == "gamma0":
        g = np.zeros(p)
    if which == "beta0":
        b = np.zeros(p)
    psi = oracle.evolve(n, cost, g, b)
    ps, norm = oracle.success_prob(n, cost, psi)
    assert abs(ps - sol / 2 ** n) < 1e-14
    assert abs(norm - 1) < 1e-13


def test_norm_and_flip_symmetry_of_state():
    """Unitary layers keep the norm; U_C, U_B and |+> all commute with the global
    flip, so psi(x) = psi(not x) (Sec. 2.2)."""
    n, k, m, p = 12, 3, 24, 5
    var, neg, cost = _sat_inst("sym", n, k, m)
    g, b = gen.linear_ramp(p)
    psi = oracle.evolve(n, cost, g, b)
    _, norm = oracle.success_prob(n, cost, psi)
    assert abs(norm - 1) < 1e-13
    x = np.arange(1 << n)
    assert np.max(np.abs(psi - psi[(~x) & ((1 << n) - 1)])) < 1e-15


def test_beta_half_pi_layer_keeps_psucc():
    """exp(i pi/2 sum_j X_j) = i^n X^{(x)n}: on a flip-symmetric state a layer with
    beta = pi/2 and gamma = 0 is a global phase, so p_succ is unchanged."""
    n, k, m = 9, 3, 18
    var, neg, cost = _sat_inst("halfpi", n, k, m)
    g, b = gen.linear_ramp(3)
    p1, _ = oracle.success_prob(n, cost, oracle.evolve(n, cost, g, b))
    p2, _ = oracle.success_prob(n, cost, oracle.evolve(n, cost, list(g) + [0.0], list(b) + [math.pi / 2]))
    assert abs(p1 - p2) < 1e-14


def test_sign_and_conjugation_relations():
    """Complex conjugation maps (g, b, s) to (-g, -b, s); flipping the mixer sign
    is b -> -b.  Both leave or map p_succ as stated."""
    n, k, m, p = 8, 3, 16, 3
    var, neg, cost = _sat_inst("conj", n, k, m)
    g, b = gen.linear_ramp(p)
    ps = lambda gg, bb, s: oracle.success_prob(n, cost, oracle.evolve(n, cost, gg, bb, s))[0]
    assert abs(ps(g, b, 1) - ps(-g, -b, 1)) < 1e-14
    assert abs(ps(g, b, -1) - ps(g, -b, 1)) < 1e-14


def test_success_prob_summation():
    """p_succ and norm against an exactly rounded sum (math.fsum)."""
    n, k, m = 11, 3, 22
    var, neg, cost = _sat_inst("sum", n, k, m)
    psi = oracle.evolve(n, cost, *gen.linear_ramp(4))
    ps, norm = oracle.success_prob(n, cost, psi)
    w = np.abs(psi) ** 2
    assert abs(ps - math.fsum(w[cost == 0])) < 1e-15
    assert abs(norm - math.fsum(w)) < 1e-14


# --------------------------------------------------------------------------
# Gradient


def test_grad_n1_analytic():
    """n = 1, C = [0, 1], one layer: p = (1 + sin 2b sin g)/2, so
    dp/dg = sin(2b) cos(g)/2 and dp/db = cos(2b) sin(g)."""
    cost = np.array([0, 1], dtype=np.uint16)
    g, b = 0.7, 0.3
    ps, dg, db = oracle.grad(1, cost, [g], [b])
    assert abs(ps - _closed_form_n1(g, b, 1)) < 1e-15
    assert abs(dg[0] - 0.5 * math.sin(2 * b) * math.cos(g)) < 1e-14
    assert abs(db[0] - math.cos(2 * b) * math.sin(g)) < 1e-14


@pytest.mark.parametrize("sign", [1, -1])
def test_grad_central_differences(sign):
    n, k, m, p = 9, 3, 18, 4
    var, neg, cost = _sat_inst("fd", n, k, m)
    g, b = gen.linear_ramp(p)
    ps, dg, db = oracle.grad(n, cost, g, b, sign)
    f = lambda gg, bb: oracle.success_prob(n, cost, oracle.evolve(n, cost, gg, bb, sign))[0]
    assert abs(ps - f(g, b)) < 1e-15
    h = 1e-5
    for l in range(p):
        e = np.zeros(p)
        e[l] = h
        fd_g = (f(g + e, b) - f(g - e, b)) / (2 * h)
        fd_b = (f(g, b + e) - f(g, b - e)) / (2 * h)
        scale = max(abs(fd_g), abs(fd_b), 1e-3)
        assert abs(dg[l] - fd_g) < 1e-8 * scale + 1e-11
        assert abs(db[l] - fd_b) < 1e-8 * scale + 1e-11


def test_grad_beta_vanishes_at_gamma_zero():
    """With gamma = 0 the state stays |+> up to a phase for every beta, so p_succ
    does not depend on beta: dp/dbeta_l = 0."""
    n, k, m, p = 8, 3, 16, 3
    var, neg, cost = _sat_inst("g0", n, k, m)
    _, dg, db = oracle.grad(n, cost, np.zeros(p), np.array([0.3, -0.2, 0.9]))
    assert np.max(np.abs(db)) < 1e-14
    assert np.max(np.abs(dg)) > 1e-6  # gamma direction is not flat in general
