"""The C ABI library: it loads, exports every function that include/qsim.h declares, and its host-only
entry points (planning, validation, schedule description, index maps) behave. No GPU needed."""
import ctypes
import random
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsim.h")


@pytest.fixture(scope="module")
def q():
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsim_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("qsim_plan", "qsim_forward", "qsim_backward", "qsim_plan_destroy", "qsim_last_error",
                 "qsim_sync_status", "qsim_expval_z"):
        assert must in names


def test_library_exports_every_declared_symbol(q):
    from paper_2404_09213_gb300 import _lib
    L = ctypes.CDLL(_lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in qsim.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature in the binding"


def test_struct_sizes_match_header(q):
    from paper_2404_09213_gb300 import _lib
    assert ctypes.sizeof(_lib.QsimGate) == 24
    assert ctypes.sizeof(_lib.QsimPlanOpts) == 80
    assert ctypes.sizeof(_lib.QsimPlanInfo) == 48


@pytest.mark.parametrize("gates,n,code", [
    ([W.gate(9, (0,))], 2, -4),                                 # unknown type
    ([W.gate(W.RX, (2,), param=0)], 2, -2),                      # qubit out of range
    ([W.gate(W.CNOT, (1,), (1,))], 2, -2),                       # control == target
    ([W.gate(W.RY, (0,))], 2, -3),                               # rotation without parameter
    ([W.gate(W.H, (0,), param=3)], 2, -3),                       # fixed gate with a parameter
    ([W.gate(W.RX, (0, 1), param=0)], 2, -2),                    # stray second target
    ([W.gate(W.RZ, (0,), param=1 << 24)], 2, -3),                # parameter index beyond any buffer
    ([W.gate(W.RZ, (0,), param=-2 - (1 << 20))], 2, -3),         # input column beyond any buffer
    ([W.gate(W.RZ, (0,), param=-(1 << 31))], 2, -3),
    ([], 0, -9),                                                 # n_qubits out of range
    ([], 35, -9),
])
def test_validation_errors(q, gates, n, code):
    with pytest.raises(q.QsimError) as e:
        q.Plan(gates, n)
    assert e.value.code == code
    assert str(e.value)


def test_backward_without_forward_is_rejected(q):
    p = q.Plan(W.ring_ansatz(3, 1), 3)
    from paper_2404_09213_gb300 import _lib
    rc = _lib.lib().qsim_backward(p._h, ctypes.c_void_p(16), None, None, None)
    assert rc == -5 and b"without a preceding forward" in _lib.lib().qsim_last_error()


def test_plan_info_and_defaults(q):
    p = q.Plan(W.ring_ansatz(20, 10), 20)
    inf = p.info()
    assert (inf["n_qubits"], inf["n_gates"], inf["n_params"], inf["n_inputs"], inf["k"]) == (20, 620, 400, 20, 12)
    p2 = q.Plan(W.ring_ansatz(20, 2), 20, dtype="c128")
    assert p2.info()["k"] == 11
    p3 = q.Plan(W.ring_ansatz(5, 2), 5, mode="per_gate")
    assert p3.info()["n_passes"] == len(W.ring_ansatz(5, 2))


@pytest.mark.parametrize("gates,n,kw", [
    (W.ring_ansatz(10, 2), 10, {"k": 8}),
    (W.hea_cz_ansatz(9, 2), 9, {"k": 7, "contiguous_bits": 2}),
    (W.ring_ansatz(4, 2), 4, {"dtype": "c128"}),
    ([W.gate(W.H, (0,)), W.gate(W.X, (1,)), W.gate(W.CZ, (2,), (0,)), W.gate(W.RX, (1,), param=0)], 3, {"k": 3, "contiguous_bits": 1}),
])
def test_specialised_kernels_compile_on_host(q, gates, n, kw):
    # NVRTC runs without a GPU: the generated pass kernels must compile for sm_103a
    p = q.Plan(gates, n, **kw)
    src = p.kernel_source()
    assert src.count('extern "C" __global__') >= 2
    p.compile_kernels()


@pytest.mark.parametrize("gates,n,kw", [
    # packed backward with CZ runs: factor tables (with thread factors and CZ signs) next to in-register
    # butterflies for runs wider than a tile's 8 threads, and 4 tiles per 32-thread CTA
    (W.hea_cz_ansatz(10, 3), 10, {"k": 8}),
    # complex128 tables (two values per entry) and the product prefix
    (W.hea_cz_ansatz(9, 2), 9, {"k": 9, "dtype": "c128"}),
    # 32-thread tiles: every run of the ring ansatz from a table
    (W.ring_ansatz(12, 3), 12, {"k": 10}),
])
def test_diagonal_tables_and_grouped_tiles_compile_on_host(q, gates, n, kw):
    p = q.Plan(gates, n, **kw)
    src = p.kernel_source()
    assert "build_tables" in src
    p.compile_kernels()


def test_diagonal_runs_with_thread_factors_compile_on_host(q):
    # runs of RZ and CZ on thread and register bits: table entries times a thread-uniform factor and
    # signed by register-thread CZs, and the in-register butterfly for the widest runs
    rng = random.Random(0)
    n = 10
    gates = [W.gate(W.H, (i,)) for i in range(n)]
    for _ in range(120):
        r = rng.random()
        if r < 0.5:
            gates.append(W.gate(W.RZ, (rng.randrange(n),), param=rng.randrange(6)))
        elif r < 0.7:
            c, t = rng.sample(range(n), 2)
            gates.append(W.gate(W.CZ, (t,), (c,)))
        elif r < 0.85:
            gates.append(W.gate(W.RY, (rng.randrange(n),), param=rng.randrange(6)))
        else:
            c, t = rng.sample(range(n), 2)
            gates.append(W.gate(W.CNOT, (t,), (c,)))
    p = q.Plan(gates, n, k=9)
    src = p.kernel_source()
    assert "qj::cmul(fr, fi, tr, ti)" in src and "fr = -fr" in src and "T dr[" in src
    p.compile_kernels()


def test_pauli_frame_kernels_take_the_tangent_form_only(q):
    # with a Pauli frame no rotation reads its per-sample form: the cotangent branch is compiled out
    gates = W.ring_ansatz(10, 2)
    src0 = q.Plan(gates, 10, k=8, pauli_frame=False).kernel_source()
    src1 = q.Plan(gates, 10, k=8, pauli_frame=True).kernel_source()
    assert "c.fm[" in src0 and "c.fm[" not in src1
    q.Plan(gates, 10, k=8, pauli_frame=True).compile_kernels()
    with pytest.raises(q.QsimError):
        q.Plan(gates, 10, mode="per_gate", pauli_frame=True)


def test_landscape_and_autotune_reject_bad_arguments_on_the_host(q):
    # argument checks run before any device work, so they can be exercised without a GPU
    import ctypes
    from paper_2404_09213_gb300 import _lib
    L = _lib.lib()
    gates = W.sel_ansatz(3, 1, encode=True)                      # has input-encoded gates
    arr = q.gate_structs(gates)
    dummy = ctypes.c_void_p(16)
    opts = _lib.QsimPlanOpts()
    L.qsim_default_opts(ctypes.byref(opts))
    rc = L.qsim_landscape(arr, len(gates), 3, ctypes.byref(opts), dummy, dummy, 4, dummy, dummy, None, None)
    assert rc == -3 and b"input-encoded" in L.qsim_last_error()
    rc = L.qsim_landscape(arr, len(gates), 3, ctypes.byref(opts), dummy, dummy, 0, dummy, dummy, None, None)
    assert rc == -1
    opts.mode = 1
    rc = L.qsim_autotune(arr, len(gates), 3, 4, 1, 1, ctypes.byref(opts), None, None)
    assert rc == -1 and b"fused" in L.qsim_last_error()
    opts.mode = 0
    rc = L.qsim_autotune(arr, len(gates), 3, 0, 1, 1, ctypes.byref(opts), None, None)
    assert rc == -1
    k = (ctypes.c_int32 * 1)()
    rc = L.qsim_multi_autotune(None, None, None, 0, 4, 1, 1, None, k, None)
    assert rc == -1


def test_batch_times_state_size_is_bounded(q):
    # batch x 2^n above 2^40 amplitudes is refused before any device work (no GPU needed)
    import ctypes
    from paper_2404_09213_gb300 import _lib
    L = _lib.lib()
    p = q.Plan(W.ring_ansatz(34, 1), 34)
    dummy = ctypes.c_void_p(256)
    rc = L.qsim_forward(p._h, dummy, dummy, 1 << 7, None, dummy, dummy, None)
    assert rc == -9 and "2^40" in L.qsim_last_error().decode()
    rc = L.qsim_expval_z(dummy, 1 << 7, 34, 0, dummy, None)
    assert rc == -9


def test_multi_plan_host_side(q):
    # planning several circuits and their buffer offsets need no GPU; errors name the circuit
    circuits = [(W.ring_ansatz(3, 1), 3), (W.hea_cz_ansatz(5, 2), 5), ([W.gate(W.H, (0,))], 1)]
    mp = q.MultiPlan(circuits)
    off = mp.offsets(4)
    n_par = [W.count_params(g) for g, _ in circuits]
    n_in = [W.count_inputs(g) for g, _ in circuits]
    assert list(off["params"]) == list(np.cumsum([0] + n_par))
    assert list(off["inputs"]) == list(4 * np.cumsum([0] + n_in))
    assert list(off["states"]) == list(4 * np.cumsum([0] + [2 ** n for _, n in circuits]))
    assert list(off["z"]) == list(4 * np.cumsum([0] + [n for _, n in circuits]))
    with pytest.raises(q.QsimError, match="circuit 1"):
        q.MultiPlan([(W.ring_ansatz(3, 1), 3), ([W.gate(W.RX, (7,), param=0)], 3)])
    with pytest.raises(q.QsimError, match="30 qubits"):
        q.MultiPlan([(W.ring_ansatz(31, 1), 31)])
    with pytest.raises(q.QsimError):
        q.MultiPlan(circuits, ks=[4, 0, 1])                      # per-circuit k outside [1, max]
