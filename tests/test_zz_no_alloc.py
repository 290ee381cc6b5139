"""The allocation-free p_succ entry point, called through the C ABI.

Callers that cannot allocate device memory when they need the result (hosts
whose allocator owns the device, paths that must not risk cudaMalloc's implicit
synchronisation) use
qaoa_success_prob_noalloc, whose scratch is a fixed array inside the library.
It must give the same numbers as qaoa_success_prob, on consecutive calls too
(the shared array keeps the previous call's contents).  This file is collected
last so that a failure here comes after every other test has run.
"""
import ctypes

import pytest

from paper_2401_02852_gb300 import instances as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2401_02852_gb300 import api  # noqa: E402
from paper_2401_02852_gb300._lib import load  # noqa: E402

REL_TOL = 1e-12  # same kernels and block count: the results agree to rounding of the final sums


def _noalloc(n, cost, state, dtype):
    ps, nm = ctypes.c_double(), ctypes.c_double()
    rc = load().qaoa_success_prob_noalloc(n, api._ptr(cost), api._ptr(state), api.dtype_code(dtype),
                                          ctypes.byref(ps), ctypes.byref(nm), api._stream(None))
    return rc, ps.value, nm.value


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_matches_success_prob_on_consecutive_calls(dtype):
    cases = []
    for n, p, idx in ((21, 4, 0), (17, 7, 1)):
        inst = gen.raw_instance("noalloc", n, 5, 8.0, idx)
        cost, _, _ = api.cost_table(inst)
        state, _, _ = api.evolve(n, cost, inst.m, *gen.linear_ramp(p), dtype)
        cases.append((n, cost, state, api.success_prob(n, cost, state)))
    for _ in range(2):  # two calls in a row on each state, alternating states
        for n, cost, state, (ref_ps, ref_nm) in cases:
            rc, ps, nm = _noalloc(n, cost, state, dtype)
            assert rc == 0, load().qaoa_last_error()
            assert abs(ps - ref_ps) <= REL_TOL * abs(ref_ps)
            assert abs(nm - ref_nm) <= REL_TOL * abs(ref_nm)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_grid_stride_matches_oracle(dtype):
    """States of 2^24 and 2^26 amplitudes (each block of the fixed grid strides
    over several chunks) against the FP64 oracle's sums of the same state:
    complex64 within 8 u = 4.8e-7 relative (pairwise FP32 sums of a thread's
    32 terms, FP64 above), complex128 within 1e-12."""
    import numpy as np

    import oracle

    tol = 8 * 2.0 ** -24 if dtype == "c64" else 1e-12
    for n, p in ((24, 3), (26, 2)):
        inst = gen.raw_instance("noalloc-big", n, 5, 8.0, 0)
        cost, _, _ = api.cost_table(inst)
        state, _, _ = api.evolve(n, cost, inst.m, *gen.linear_ramp(p), dtype)
        cost_o, _, _ = oracle.cost_table(n, inst.var, inst.neg)
        ref_ps, ref_nm = oracle.success_prob(n, cost_o, state.cpu().numpy().astype(np.complex128))
        for _ in range(2):
            rc, ps, nm = _noalloc(n, cost, state, dtype)
            assert rc == 0, load().qaoa_last_error()
            assert abs(ps - ref_ps) <= tol * ref_ps + 1e-300 and abs(nm - ref_nm) <= tol * ref_nm
        del state, cost
        torch.cuda.empty_cache()


def test_noalloc_rejects_out_of_range_size():
    cost = torch.zeros(16, dtype=torch.uint8, device="cuda")
    state = torch.zeros(16, dtype=torch.complex64, device="cuda")
    rc, _, _ = _noalloc(40, cost, state, "c64")
    assert rc == -2 and b"outside" in load().qaoa_last_error()
