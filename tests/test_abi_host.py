"""Host-only checks of the C ABI: the library builds, loads and exports every
function that include/qaoa.h declares; host logic (planning, validation) runs
without a GPU.  No call here launches device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2401_02852_gb300 import _build, _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "qaoa.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("naesat_cost_table", "qaoa_evolve", "qaoa_success_prob", "qaoa_grad", "qaoa_serve_submit",
                     "qaoa_serve_poll"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding binds exactly the declared set
    assert sorted(_lib.SIGNATURES) == names


def test_version_and_kernel_names(lib):
    assert lib.qaoa_version() >= 100
    names = [lib.qaoa_kernel_name(i).decode() for i in range(16)]
    assert "pass_low" in names and "cost_table" in names


def _plan(lib, n, dtype, flags=0):
    lo = (ctypes.c_int * 8)()
    bits = (ctypes.c_int * 8)()
    row = (ctypes.c_int * 8)()
    k = lib.qaoa_plan(n, dtype, flags, lo, bits, row)
    return k, [(lo[i], bits[i], row[i]) for i in range(max(k, 0))]


@pytest.mark.parametrize("dtype,T,G,rows", [(0, 13, 9, (4, 5)), (1, 12, 8, (4,))])
def test_plan_covers_every_qubit_once(lib, dtype, T, G, rows):
    """Every qubit is mixed by exactly one pass; high groups span T - row bits
    (complex64 also takes 256-byte rows of 5 bits, groups of 8), with no more
    passes than groups of the widest size need."""
    for n in range(T + 1, 33):
        k, passes = _plan(lib, n, dtype)
        assert k == len(passes) >= 2
        assert k - 1 == -(-(n - T) // G)
        mixed = list(range(passes[0][1]))
        assert passes[0] == (0, T, T)
        for lo, bits, row in passes[1:]:
            g = T - row
            assert row in rows and lo >= row and lo + g <= n and 1 <= bits <= g
            mixed += list(range(lo + g - bits, lo + g))  # the top `bits` of the group
        assert sorted(mixed) == list(range(n)), (n, passes)
    if dtype == 0:  # n = 30: rows of 16 for bits 13..21, of 32 for bits 22..29
        assert _plan(lib, 30, dtype)[1] == [(0, 13, 13), (13, 9, 4), (22, 8, 5)]


def test_plan_rejects_out_of_range(lib):
    assert lib.qaoa_plan(50, 0, 0, None, None, None) == _lib_code("ERANGE")
    assert lib.qaoa_plan(20, 7, 0, None, None, None) == _lib_code("EINVAL")
    assert b"dtype" in lib.qaoa_last_error()


def _lib_code(name):
    return {v: k for k, v in _lib.ERRORS.items()}[name]


def test_argument_validation_precedes_device_work(lib):
    """Invalid calls return their error from host validation, before any CUDA call."""
    assert lib.naesat_cost_table(None, None, None, None, None) == _lib_code("EINVAL")
    var = np.array([[0, 0, 1]], dtype=np.int32)  # repeated variable
    neg = np.zeros((1, 3), dtype=np.uint8)
    inst = _lib.NaesatInstance(4, 1, 3, var.ctypes.data, neg.ctypes.data)
    assert lib.naesat_cost_table(ctypes.byref(inst), ctypes.c_void_p(1), None, None, None) == _lib_code("EINVAL")
    assert b"repeated" in lib.qaoa_last_error()
    inst = _lib.NaesatInstance(40, 1, 3, var.ctypes.data, neg.ctypes.data)
    assert lib.naesat_cost_table(ctypes.byref(inst), ctypes.c_void_p(1), None, None, None) == _lib_code("ERANGE")
    inst = _lib.NaesatInstance(20, 8192, 3, var.ctypes.data, neg.ctypes.data)  # one past the clause limit
    assert lib.naesat_cost_table(ctypes.byref(inst), ctypes.c_void_p(1), None, None, None) == _lib_code("ERANGE")
    assert lib.qaoa_evolve(20, ctypes.c_void_p(1), 8192, 0, None, None, 0, 0, ctypes.c_void_p(1),
                           None, None, None) == _lib_code("ERANGE")
    g = np.array([0.1, float("nan")])
    assert lib.qaoa_evolve(20, ctypes.c_void_p(1), 10, 2, g.ctypes.data, g.ctypes.data, 0, 0, ctypes.c_void_p(1),
                           None, None, None) == _lib_code("EINVAL")
    assert lib.qaoa_evolve(20, ctypes.c_void_p(1), 10, 1, g.ctypes.data, g.ctypes.data, 9, 0, ctypes.c_void_p(1),
                           None, None, None) == _lib_code("EINVAL")
    assert lib.qaoa_grad(20, ctypes.c_void_p(1), 10, 0, None, None, 0, 0, ctypes.c_void_p(1), ctypes.c_void_p(1),
                         None, None, None, None) == _lib_code("EINVAL")


def _schedule(lib, n, p, dtype, flags=0):
    cap = 8 * p + 8
    idx, lay, mod = (ctypes.c_int * cap)(), (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
    k = lib.qaoa_pass_schedule(n, p, dtype, flags, cap, idx, lay, mod)
    return [(idx[i], lay[i], mod[i]) for i in range(k)]


@pytest.mark.parametrize("dtype,T", [(0, 13), (1, 12)])
@pytest.mark.parametrize("p", [0, 1, 2, 5, 10])
@pytest.mark.parametrize("z2", [False, True])
def test_schedule_applies_each_layer_in_order(lib, dtype, T, p, z2):
    """Replays the launch sequence symbolically: every layer applies its phase
    once, then mixes every qubit exactly once, before the next layer's phase
    (the layer product of the QAOA output state).  In the halved plan the low
    pass mixes qubits [0, T - 1) and the top qubit n - 1 (the mirror)."""
    flags = 2 if z2 else 0
    for n in (T + 1, 22, 30, 32):
        _, passes = _plan(lib, n, dtype, flags)

        def qubits(i):
            if i == 0:
                return list(range(T - 1)) + [n - 1] if z2 else list(range(T))
            lo, bits, row = passes[i]
            g = T - row
            return list(range(lo + g - bits, lo + g))

        events = []
        sched = _schedule(lib, n, p, dtype, flags)
        for pi, l, mode in sched:
            if mode in (0, 3):
                events.append(("phase", l, None))
            if p > 0:
                events += [("mix", l, q) for q in qubits(pi)]
            if mode == 2:
                assert pi != 0  # the low pass never fuses
                events.append(("phase", l + 1, None))
                events += [("mix", l + 1, q) for q in qubits(pi)]
        if p == 0:
            assert events == [("phase", 0, None)]
            continue
        if len(passes) >= 3:  # every layer boundary fuses
            assert len(sched) == p * (len(passes) - 1) + 1
        else:  # one high group: the boundaries on it fuse, those on the low pass do not
            assert len(sched) == 2 * p - p // 2
        layer, seen = -1, None
        for kind, l, q in events:
            if kind == "phase":
                assert l == layer + 1 and (seen is None or sorted(seen) == list(range(n)))
                layer, seen = l, []
            else:
                assert l == layer and q not in seen
                seen.append(q)
        assert layer == p - 1 and sorted(seen) == list(range(n))


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,p", [(13, 1), (13, 4), (20, 3), (22, 20), (30, 10), (32, 5)])
def test_adjoint_schedule_undoes_each_layer_in_reverse(lib, dtype, n, p):
    """Replays the backward sweep: layers p-1 .. 0 in turn; every pass undoes
    each layer's butterflies exactly once, and the layer's phase goes after all
    of them (mode 1 or 2 on its last pass); a fused launch (mode 2) goes on to
    undo layer l - 1 on the same group, so that layer skips it."""
    cap = 8 * p + 8
    idx, lay, mod = (ctypes.c_int * cap)(), (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
    k = lib.qaoa_adjoint_schedule(n, p, dtype, cap, idx, lay, mod)
    assert k > 0
    seq = [(idx[i], lay[i], mod[i]) for i in range(k)]
    n_passes = max(s[0] for s in seq) + 1
    undone = {l: [] for l in range(p)}
    phase_done = []
    for pi, l, mode in seq:
        assert l not in phase_done and all(x in phase_done for x in range(l + 1, p))
        undone[l].append(pi)
        if mode in (1, 2):
            assert sorted(undone[l]) == list(range(n_passes))  # the whole layer first
            phase_done.append(l)
        if mode == 2:
            assert pi != 0 and l >= 1
            undone[l - 1].append(pi)
    assert phase_done == list(range(p - 1, -1, -1))
    if n_passes >= 3:  # every boundary fuses: one launch saved per boundary
        assert k == n_passes + (p - 1) * (n_passes - 1)
    else:
        assert k == 2 * p


def test_sampling_validation_precedes_device_work(lib):
    """qaoa_sample / qaoa_running_time reject bad arguments on the host."""
    one = ctypes.c_void_p(1)
    rt = ctypes.c_int64()
    assert lib.qaoa_sample(20, one, 0, 0, 16, one, None, None) == _lib_code("EINVAL")          # no output
    assert lib.qaoa_sample(20, one, 0, 0, 0, one, one, None) == _lib_code("ERANGE")            # k = 0
    assert lib.qaoa_sample(33, one, 0, 0, 16, one, one, None) == _lib_code("ERANGE")           # n > 32
    assert lib.qaoa_sample(1, one, 0, 2, 16, one, one, None) == _lib_code("ERANGE")            # halved needs n >= 2
    assert lib.qaoa_sample(20, one, 5, 0, 16, one, one, None) == _lib_code("EINVAL")           # dtype
    assert lib.qaoa_sample(20, one, 0, 0x100, 16, one, one, None) == _lib_code("EINVAL")       # unknown flag
    assert lib.qaoa_sample(20, None, 0, 0, 16, one, one, None) == _lib_code("EINVAL")          # no state
    assert lib.qaoa_running_time(20, None, one, 0, 0, 16, one, ctypes.byref(rt), None, None) == _lib_code("EINVAL")
    assert lib.qaoa_running_time(20, one, one, 0, 0, 16, one, None, None, None) == _lib_code("EINVAL")
    assert lib.qaoa_running_time_batch(0, 20, one, one, 0, 0, 16, one, ctypes.byref(rt), None) == _lib_code("ERANGE")
    assert lib.qaoa_adjoint_schedule(20, 0, 0, 0, None, None, None) == _lib_code("EINVAL")
