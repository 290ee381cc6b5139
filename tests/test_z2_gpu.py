"""The halved state (QAOA_Z2_HALF): NAE's global-flip symmetry (Sec. 2.2) gives
psi(x) = psi(not x), so the library may store only x < 2^(n-1).  The halved
evolution must reproduce the full one: the stored half equals the first half of
the full state and p_succ / norm agree."""
import numpy as np
import pytest

import oracle
from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api  # noqa: E402
from paper_2401_02852_gb300._lib import Z2_HALF, QaoaError  # noqa: E402


def _inst(n, idx, k=5, tag="z2"):
    for a in range(1000):
        inst = gen.raw_instance(tag, n, k, 8.0, idx, a)
        full, sol, _ = api.cost_table(inst)
        if sol:
            return inst, full
    raise RuntimeError


@pytest.mark.parametrize("n", [6, 9, 14, 17, 22])
def test_half_table_is_first_half(n):
    inst = gen.raw_instance("z2-tab", n, 3 if n < 10 else 5, 8.0, 0)
    full, sol, mx = api.cost_table(inst)
    half, hsol, hmx = api.cost_table_half(inst)
    assert torch.equal(half, full[: 1 << (n - 1)])
    assert (hsol, hmx) == (sol, mx)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,p,sign,kind", [(14, 3, 0, "ramp"), (15, 1, 1, "ramp"), (17, 4, 0, "steep"),
                                           (20, 2, 1, "steep"), (23, 3, 0, "ramp"), (16, 0, 0, "ramp"),
                                           (22, 5, 0, "ramp")])
def test_halved_evolution_matches_full(dtype, n, p, sign, kind):
    inst, full = _inst(n, p)
    half = full[: 1 << (n - 1)].contiguous()
    g, b = gen.linear_ramp(p)
    if kind == "steep":
        b = np.where(np.arange(p) % 2 == 0, 1.2, -1.35)
    s_full, ps_full, nm_full = api.evolve(n, full, inst.m, g, b, dtype, flags=sign)
    s_half, ps_half, nm_half = api.evolve(n, half, inst.m, g, b, dtype, flags=sign | Z2_HALF)
    assert s_half.numel() == 1 << (n - 1)
    if dtype == "c128":
        assert torch.max(torch.abs(s_half - s_full[: 1 << (n - 1)])).item() < 1e-13
        assert abs(ps_half - ps_full) <= 1e-12 * ps_full and abs(nm_half - nm_full) < 1e-12
    else:
        amp = torch.max(torch.abs(s_full)).item()
        assert torch.max(torch.abs(s_half - s_full[: 1 << (n - 1)])).item() <= 1e-6 * (1 + n * p) * amp
        assert abs(ps_half - ps_full) <= 1e-5 * ps_full and abs(nm_half - 1) < 1e-6
    if n <= 20:  # and against the oracle
        ref = oracle.cost_table(n, inst.var, inst.neg)[0]
        rps, _ = oracle.success_prob(n, ref, oracle.evolve(n, ref, g, b, -1 if sign else 1))
        assert abs(ps_half - rps) <= (1e-10 if dtype == "c128" else 1e-4) * rps


def test_halved_batch():
    n, p = 16, 4
    insts = [_inst(n, i, tag="z2b")[0] for i in range(4)]
    halves = torch.stack([api.cost_table_half(x)[0] for x in insts])
    g, b = gen.linear_ramp(p)
    st, ps, nm = api.evolve_batch(n, halves, insts[0].m, g, b, "c64", flags=Z2_HALF)
    assert st.shape == (4, 1 << (n - 1))
    for i, inst in enumerate(insts):
        full, _, _ = api.cost_table(inst)
        _, p1, _ = api.evolve(n, full, inst.m, g, b, "c64")
        assert abs(ps[i] - p1) <= 1e-5 * p1


def test_halved_state_rejects_small_n():
    inst = gen.raw_instance("z2-small", 12, 3, 2.0, 0)
    half, _, _ = api.cost_table_half(inst)
    with pytest.raises(QaoaError):
        api.evolve(12, half, inst.m, *gen.linear_ramp(2), "c64", flags=Z2_HALF)
