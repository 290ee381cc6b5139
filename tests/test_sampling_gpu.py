"""Bitstring draws and running times on the GPU against the FP64 oracle.

The sampler's input is a seeded synthetic state from the generator module (or
an evolution that both sides compute themselves), the uniforms are shared, and
the draws must agree one by one.  A draw may differ only where its uniform
lies within rounding of a step of the cumulative distribution (the two sides
sum in different orders); each such case is checked to be one.
"""
import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api  # noqa: E402
from paper_2401_02852_gb300._lib import Z2_HALF  # noqa: E402


# A draw may differ from the oracle's only where its uniform lies within about
# 2^-40 F_total of a step of the cumulative distribution: the sampler's integer
# weights are exact to 2^-44 of a 2^13-amplitude group's largest probability,
# and the oracle's running FP64 sum is within about sqrt(N) 2^-53 F_total of the
# exact one for these states.  The window is 1e-11 F_total around a step of the
# exact distribution (a long-double running sum).
TIE_REL = 1e-11


def _exact_cdf(psi):
    p = np.abs(psi.astype(np.complex128)) ** 2
    return np.cumsum(p.astype(np.longdouble))


def _near_step(F, u, x, rel=TIE_REL):
    """True when u F_total is within `rel` F_total of F(x - 1) or F(x) (a tie the
    summation order may break either way)."""
    t = np.longdouble(u) * F[-1]
    lo = F[x - 1] if x > 0 else np.longdouble(0.0)
    return float(min(abs(t - lo), abs(t - F[x]))) <= rel * float(F[-1])


def _check_draws(psi, u, got, want):
    bad = np.flatnonzero(got != want)
    if bad.size:
        F = _exact_cdf(psi)
        for j in bad:
            assert _near_step(F, u[j], int(want[j])) and _near_step(F, u[j], int(got[j])), (j, got[j], want[j])
    assert bad.size <= max(2, u.size // 1000)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
@pytest.mark.parametrize("n,sparsity", [(5, 0.0), (12, 0.3), (14, 0.0), (17, 0.6), (20, 0.0), (24, 0.0),
                                        (26, 0.5)])
def test_draws_match_oracle(n, sparsity, dtype):
    psi = gen.random_state("gpu-draw", n, n, sparsity=sparsity).astype(dtype)
    u = np.concatenate([gen.uniforms("gpu-draw", 3000, n), [0.0, 0.5, 1.0 - 2.0 ** -53]])
    want = oracle.sample(n, psi.astype(np.complex128), u)
    got = api.sample(n, torch.from_numpy(psi).cuda(), u).cpu().numpy().astype(np.uint64)
    _check_draws(psi, u, got, want)
    p = np.abs(psi.astype(np.complex128)) ** 2
    assert np.all(p[got.astype(np.int64)] > 0)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_halved_state_draws(dtype):
    """Halved state (flip-symmetric psi stored for x with bit n-1 clear): a draw
    with u < 1/2 is the half's draw at 2u, one with u >= 1/2 the complement of
    the half's draw at 2u - 1."""
    n = 15
    half = gen.random_state("gpu-z2", n - 1, 0).astype(dtype).astype(np.complex128)
    full = np.concatenate([half, half[::-1]]) / np.sqrt(2)  # psi(not x) = psi(x)
    u = gen.uniforms("gpu-z2", 4000, 0)
    got = api.sample(n, torch.from_numpy(half.astype(dtype)).cuda(), u, flags=Z2_HALF).cpu().numpy().astype(np.uint64)
    lo = u < 0.5
    want = np.empty_like(got)
    want[lo] = oracle.sample(n - 1, half, 2 * u[lo])
    want[~lo] = (~oracle.sample(n - 1, half, 2 * u[~lo] - 1)) & np.uint64((1 << n) - 1)
    bad = np.flatnonzero(got != want)
    assert bad.size <= 4, bad
    if bad.size:  # each difference is a tie of the half's distribution at 2u or 2u - 1
        F = _exact_cdf(half)
        for j in bad:
            uj = 2 * u[j] if lo[j] else 2 * u[j] - 1
            mask = np.uint64((1 << (n - 1)) - 1)
            wx, gx = int(want[j] & mask), int(got[j] & mask)
            if not lo[j]:
                wx, gx = int(~want[j] & mask), int(~got[j] & mask)
            assert _near_step(F, uj, wx) and _near_step(F, uj, gx), (j, got[j], want[j])
    # every draw has the probability the full state gives it
    assert np.all(np.abs(full[got.astype(np.int64)]) > 0)


def test_frequencies_match_the_born_rule():
    n, draws = 6, 60000
    psi = gen.random_state("gpu-born", n, 0)
    xs = api.sample(n, torch.from_numpy(psi.astype(np.complex64)).cuda(), gen.uniforms("gpu-born", draws, 0))
    counts = np.bincount(xs.cpu().numpy(), minlength=1 << n)
    _, pval = scipy.stats.chisquare(counts, draws * np.abs(psi) ** 2)
    assert pval > 1e-3


def _instance(n, idx, tag="gpu-rt"):
    inst, _ = gen.satisfiable_instance(tag, n, 5, 8.0, idx, oracle.count_solutions)
    return inst


@pytest.mark.parametrize("n,p", [(12, 3), (15, 5), (18, 2)])
def test_running_time_matches_oracle(n, p):
    g, b = gen.linear_ramp(p)
    for idx in range(4):
        inst = _instance(n, idx)
        cost_o, _, _ = oracle.cost_table(n, inst.var, inst.neg)
        psi_o = oracle.evolve(n, cost_o, g, b)
        ps, nm = oracle.success_prob(n, cost_o, psi_o)
        k = int(20 / (ps / nm)) + 1
        u = gen.uniforms("gpu-rt", k, 100 * n + idx)
        want = oracle.running_time(n, cost_o, psi_o, u)
        cost = api.cost_table(inst)[0]
        state, _, _ = api.evolve(n, cost, inst.m, g, b, "c128")
        got = api.running_time(n, cost, state, u)
        assert got == want and got >= 1, (idx, got, want)


def test_running_time_batch_equals_single():
    n, p, B = 14, 4, 6
    g, b = gen.linear_ramp(p)
    insts = [_instance(n, i, "gpu-rtb") for i in range(B)]
    costs, _, _ = api.cost_table_batch(insts)
    states, ps, nm = api.evolve_batch(n, costs, insts[0].m, g, b, "c64")
    k = 4096
    u = np.stack([gen.uniforms("gpu-rtb", k, i) for i in range(B)])
    rts = api.running_time_batch(n, costs, states, u)
    for i in range(B):
        assert rts[i] == api.running_time(n, costs[i].contiguous(), states[i].contiguous(), u[i])


def test_running_time_none_and_halved():
    """No satisfying draw among k gives 0; the halved state gives the same
    running time distribution as the full one (same p_succ)."""
    n, p = 16, 3
    g, b = gen.linear_ramp(p)
    inst = _instance(n, 7)
    cost = api.cost_table(inst)[0]
    state, _, _ = api.evolve(n, cost, inst.m, g, b, "c64")
    # a state with no mass on solutions: zero those amplitudes
    masked = torch.where(cost == 0, torch.zeros_like(state), state)
    assert api.running_time(n, cost, masked, gen.uniforms("gpu-none", 256, 0)) == 0
    half = api.cost_table_half(inst)[0]
    st_h, _, _ = api.evolve(n, half, inst.m, g, b, "c64", flags=Z2_HALF)
    runs = 400
    u = np.stack([gen.uniforms("gpu-geo", 2048, i) for i in range(runs)])
    rt_full = api.running_time_batch(n, cost.unsqueeze(0).expand(runs, -1).contiguous(),
                                     state.unsqueeze(0).expand(runs, -1).contiguous(), u)
    rt_half = api.running_time_batch(n, half.unsqueeze(0).expand(runs, -1).contiguous(),
                                     st_h.unsqueeze(0).expand(runs, -1).contiguous(), u, flags=Z2_HALF)
    cost_o, _, _ = oracle.cost_table(n, inst.var, inst.neg)
    ps_o, nm_o = oracle.success_prob(n, cost_o, oracle.evolve(n, cost_o, g, b))
    pp = ps_o / nm_o
    for rts in (rt_full, rt_half):
        assert np.all(rts >= 1)
        # geometric law: mean 1 / p_succ within 4 standard errors
        assert abs(rts.mean() - 1 / pp) < 4 * np.sqrt((1 - pp) / pp ** 2) / np.sqrt(runs)


def test_full_size_draws_satisfy_the_definition():
    """n = 30, p = 10 (the benchmark's evolution): the first satisfying draw is
    where the running time says, as the oracle evaluates C at the drawn x one
    by one, and no earlier draw satisfies."""
    n, p = 30, 10
    inst, _ = gen.satisfiable_instance("bench-n30", n, 5, 8.0, 0, lambda x: api.cost_table(x)[1])
    g, b = gen.linear_ramp(p)
    cost = api.cost_table(inst)[0]
    state, ps, nm = api.evolve(n, cost, inst.m, g, b, "c64")
    k = 4096
    u = gen.uniforms("gpu-n30", k, 0)
    xs = api.sample(n, state, u).cpu().numpy().astype(np.uint64)
    rt = api.running_time(n, cost, state, u)
    c = oracle.cost_samples(inst.var, inst.neg, xs)
    first = int(np.flatnonzero(c == 0)[0]) + 1 if np.any(c == 0) else 0
    assert rt == first and rt >= 1
    # draws are monotone in u
    order = np.argsort(u)
    assert np.all(np.diff(xs[order].astype(np.int64)) >= 0)
    del state, cost
    torch.cuda.empty_cache()


def test_sweep_reports_running_times(tmp_path):
    """The scaling sweep's plumbing: per (n, p) median 1/p_succ and median
    running time over instances, no censored instance at these sizes, the
    results resumable from their files, and the exponents fitted."""
    from paper_2401_02852_gb300 import sweep

    res = sweep.run_sweep(ns=(14, 16), ps=(1, 4), seeds=12, out_dir=str(tmp_path), log=None, running_times=True)
    for (n, p), r in res["results"].items():
        rts = np.array(r["running_times"])
        assert rts.size == 12 and np.all(rts >= 1) and r["censored_running_times"] == 0
        assert r["median_running_time"] == np.median(rts)
        assert r["inv_mean_psucc"] == pytest.approx(1.0 / np.mean(r["psucc"]))
    for p in (1, 4):
        assert "running_time_c_bits" in res["fits"][p]
    again = sweep.run_sweep(ns=(14, 16), ps=(1, 4), seeds=12, out_dir=str(tmp_path), log=None, running_times=True)
    assert again["results"][(16, 4)]["running_times"] == res["results"][(16, 4)]["running_times"]


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_uniforms_outside_the_unit_interval(dtype):
    """u <= 0 (and NaN) draw the first x of nonzero probability, u >= 1 the
    last; a state of norm zero draws 0."""
    n = 13
    psi = gen.random_state("gpu-edge", n, 0, sparsity=0.5)
    psi[:37] = 0  # the first entries hold no mass
    psi[-70:] = 0
    nz = np.flatnonzero(np.abs(psi.astype(dtype)) > 0)
    u = np.array([-0.5, -0.0, 0.0, np.nan, 1.0, 1.5, np.inf])
    got = api.sample(n, torch.from_numpy(psi.astype(dtype)).cuda(), u).cpu().numpy()
    assert list(got) == [nz[0]] * 4 + [nz[-1]] * 3
    zero = torch.zeros(1 << n, dtype=torch.complex64 if dtype == np.complex64 else torch.complex128, device="cuda")
    assert np.all(api.sample(n, zero, np.array([0.0, 0.3, 0.99])).cpu().numpy() == 0)


def test_staged_and_unstaged_prefix_agree():
    """A complex64 state at an address that is not 16-byte aligned takes the
    unstaged entry sums; both orders of work give the same draws."""
    n = 15
    psi = gen.random_state("gpu-align", n, 0, sparsity=0.3).astype(np.complex64)
    buf = torch.zeros((1 << n) + 1, dtype=torch.complex64, device="cuda")
    buf[1:] = torch.from_numpy(psi).cuda()
    aligned = torch.from_numpy(psi).cuda()
    shifted = buf[1:]
    assert shifted.data_ptr() % 16 == 8
    u = gen.uniforms("gpu-align", 5000, 0)
    assert torch.equal(api.sample(n, aligned, u), api.sample(n, shifted, u))
