"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: complex64 |dz| <= 1e-5, states <= 1e-5, gradients norm-wise relative <= 1e-4 and
elementwise <= 1e-4 max|g_ref| + 1e-7; complex128 1e-12 throughout.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_util import TOL, tensors, rounded, check_grad, random_circuit, shift_grad_strided

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def run(q, wl, dtype, mode="fused", init=None, backward=True, **kw):
    plan = q.Plan(wl.gates, wl.n, dtype=dtype, mode=mode, **kw)
    p, x, g = tensors(wl, dtype)
    states, z = plan.forward(p, x, init=init)
    out = {"states": states.cpu().numpy(), "z": z.cpu().numpy(), "plan": plan}
    if backward:
        dp, di = plan.backward(g)
        out["dp"], out["di"] = dp.cpu().numpy(), di.cpu().numpy()
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return out


# ---------------------------------------------------------------- C1 (4 qubits, batch 8, complex128)
@pytest.mark.parametrize("mode", ["fused", "per_gate"])
def test_c1_complex128(q, mode):
    wl = W.config(1)
    r = run(q, wl, "c128", mode)
    psi = oracle.simulate_kron(wl.gates, wl.n, wl.params, wl.inputs)
    np.testing.assert_allclose(r["states"], psi, atol=1e-12, rtol=0)
    zref = np.loadtxt(os.path.join(GOLDEN, "c1_z.txt"))
    np.testing.assert_allclose(r["z"], zref, atol=1e-12, rtol=0)
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out)
    check_grad(r["dp"], dp, "c128", "C1 dparams")
    check_grad(r["di"], di, "c128", "C1 dinputs")


@pytest.mark.parametrize("k", [3, 4])
def test_c1_fused_tile_sizes(q, k):
    wl = W.config(1)
    r = run(q, wl, "c128", "fused", k=k, contiguous_bits=1)
    psi = oracle.simulate_kron(wl.gates, wl.n, wl.params, wl.inputs)
    np.testing.assert_allclose(r["states"], psi, atol=1e-12, rtol=0)


# ---------------------------------------------------------------- random circuits, all gate types
CASES = []
for seed, (n, dtype, mode, k, c) in enumerate([
        (1, "c64", "fused", 1, 1), (2, "c64", "fused", 2, 1), (3, "c128", "fused", 3, 1),
        (5, "c64", "fused", 4, 2), (6, "c128", "fused", 5, 2), (7, "c64", "fused", 5, 3),
        (8, "c64", "fused", 6, 2), (9, "c128", "fused", 7, 3), (10, "c64", "fused", 8, 4),
        (10, "c64", "fused", 10, 4), (11, "c64", "fused", 7, 2), (6, "c64", "per_gate", 0, 0),
        (9, "c128", "per_gate", 0, 0), (12, "c64", "fused", 12, 4), (13, "c128", "fused", 11, 4)]):
    CASES.append((seed, n, dtype, mode, k, c))


@pytest.mark.parametrize("seed,n,dtype,mode,k,c", CASES)
def test_random_circuits(q, seed, n, dtype, mode, k, c):
    _random_case(q, seed, n, dtype, mode, k, c)


# qubits handed between the low (coalescing) index bits from pass to pass: each pass writes a new layout
@pytest.mark.parametrize("seed,n,dtype,k,c", [(20, 11, "c64", 8, 3), (21, 12, "c64", 10, 4), (22, 13, "c128", 11, 4),
                                              (23, 12, "c64", 6, 2)])
def test_random_circuits_rotating_layouts(q, seed, n, dtype, k, c):
    _random_case(q, seed, n, dtype, "fused", k, c, rotate_low_bits=True)


# without the Pauli frame (fused plans use it by default): every rotation picks its tangent or cotangent
# form per sample at run time, as the multi-circuit queue kernels do; with and without checkpoints
@pytest.mark.parametrize("seed,n,dtype,k,c,ckpt", [(30, 1, "c64", 1, 1, 0), (31, 5, "c128", 4, 2, 0),
                                                   (32, 7, "c64", 5, 3, 1), (33, 9, "c128", 7, 3, 1),
                                                   (34, 10, "c64", 8, 4, 0), (35, 12, "c64", 12, 4, 0),
                                                   (36, 11, "c64", 6, 2, 2), (37, 13, "c128", 11, 4, 1)])
def test_random_circuits_both_forms(q, seed, n, dtype, k, c, ckpt):
    _random_case(q, seed, n, dtype, "fused", k, c, pauli_frame=False, checkpoint_passes=ckpt)


# complex64 Pauli-frame plans update psi and lambda together with packed FP32x2 FMAs in the backward by
# default; the scalar variant against the oracle on the same random circuits (every gate kind)
@pytest.mark.parametrize("seed,n,k,c,ckpt", [(40, 6, 5, 2, 0), (41, 10, 8, 4, 1), (42, 12, 12, 4, 0)])
def test_random_circuits_frame_scalar_backward(q, seed, n, k, c, ckpt):
    _random_case(q, seed, n, "c64", "fused", k, c, pauli_frame=True, scalar_bwd=True, checkpoint_passes=ckpt)


# product-state prefix (on by default): every qubit's single-qubit gates before its first two-qubit gate
# become phi_q, the first pass starts from their product and their gradients come from one contraction
def _prefix_circuit(rng, n, g, n_params=6, n_inputs=3):
    """A random circuit whose qubits start with runs of every single-qubit gate kind (rotations on shared
    parameters and on input columns, H and X) before the entanglers begin."""
    head = []
    for qb in range(n):
        for _ in range(int(rng.integers(0, 4))):
            k = int(rng.choice([W.RX, W.RY, W.RZ, W.H, W.X]))
            if k in (W.RX, W.RY, W.RZ):
                p = W.input_param(int(rng.integers(0, n_inputs))) if rng.uniform() < 0.4 else int(rng.integers(0, n_params))
                head.append(W.gate(k, (qb,), param=p))
            else:
                head.append(W.gate(k, (qb,)))
    return head + random_circuit(rng, n, g, n_params, n_inputs)


@pytest.mark.parametrize("seed,n,dtype,k,c,ckpt", [(50, 3, "c64", 3, 1, 0), (51, 7, "c128", 5, 2, 1),
                                                   (52, 10, "c64", 8, 4, 1), (53, 12, "c64", 12, 4, 0),
                                                   (54, 13, "c128", 11, 4, 1), (55, 9, "c64", 6, 2, 2)])
def test_product_prefix_against_oracle(q, seed, n, dtype, k, c, ckpt):
    rng = np.random.default_rng(200 + seed)
    n_par, n_in, B = 6, 3, 3
    gates = _prefix_circuit(rng, n, 6 * n, n_par, n_in)
    params = rng.uniform(0, 2 * math.pi, n_par)
    inputs = rng.uniform(0, math.pi, (B, n_in))
    g = rng.uniform(-1, 1, (B, n))
    wl = W.Workload("pfx", n, B, dtype, gates, params, inputs, g)
    r = run(q, wl, dtype, "fused", k=k, contiguous_bits=c, checkpoint_passes=ckpt, product_prefix=True)
    assert any(r["plan"].describe()["prefix"])
    pr, ir = rounded(wl, dtype)
    psi = oracle.simulate_strided(gates, n, pr, ir)
    t = TOL[dtype]
    np.testing.assert_allclose(r["states"], psi, atol=t["state"], rtol=0)
    np.testing.assert_allclose(r["z"], oracle.expval_z(psi, n), atol=t["z"], rtol=0)
    dp, di = oracle.grad_adjoint(gates, n, pr, ir, g)
    check_grad(r["dp"], dp, dtype, "dparams")
    check_grad(r["di"], di, dtype, "dinputs")


def test_product_prefix_whole_circuit_and_initial_state(q):
    # no entangler at all: every gate is in a prefix and the single pass only writes the product state;
    # then an initial state, which the prefix cannot use (an internal plan without it runs instead)
    rng = np.random.default_rng(9)
    n, B = 8, 2
    gates = [W.gate(W.RX, (qb,), param=W.input_param(qb)) for qb in range(n)]
    gates += [W.gate(W.RY, (qb,), param=qb) for qb in range(n)] + [W.gate(W.H, (3,))]
    wl = W.Workload("prod", n, B, "c64", gates, rng.uniform(0, 2 * math.pi, n), rng.uniform(0, math.pi, (B, n)),
                    rng.uniform(-1, 1, (B, n)))
    r = run(q, wl, "c64", "fused", k=6)
    pr, ir = rounded(wl, "c64")
    psi = oracle.simulate_strided(gates, n, pr, ir)
    np.testing.assert_allclose(r["states"], psi, atol=1e-5, rtol=0)
    dp, di = oracle.grad_adjoint(gates, n, pr, ir, wl.grad_out)
    check_grad(r["dp"], dp, "c64", "dparams (product circuit)")
    check_grad(r["di"], di, "c64", "dinputs (product circuit)")
    init = rng.normal(size=(B, 2 ** n)) + 1j * rng.normal(size=(B, 2 ** n))
    init /= np.linalg.norm(init, axis=1, keepdims=True)
    r2 = run(q, wl, "c64", "fused", k=6, init=torch.tensor(init, dtype=torch.complex64, device="cuda"))
    i64 = init.astype(np.complex64).astype(complex)
    psi2 = oracle.simulate_strided(gates, n, pr, ir, init=i64)
    np.testing.assert_allclose(r2["states"], psi2, atol=1e-5, rtol=0)
    dp2, di2 = oracle.grad_adjoint(gates, n, pr, ir, wl.grad_out, init=i64)
    check_grad(r2["dp"], dp2, "c64", "dparams (initial state)")
    check_grad(r2["di"], di2, "c64", "dinputs (initial state)")


def test_product_prefix_equals_plain_plan_on_c3_ansatz(q):
    # the 14-qubit version of the 20-qubit workload: the prefix holds the RX encoding and the first layer
    wl = W.config(3, n=14, batch=4)
    a = run(q, wl, "c64", "fused", k=10, checkpoint_passes=1, product_prefix=False)
    b = run(q, wl, "c64", "fused", k=10, checkpoint_passes=1, product_prefix=True)
    assert [len(x) for x in b["plan"].describe()["prefix"]] == [3] * 14
    assert b["plan"].info()["n_passes"] <= a["plan"].info()["n_passes"]
    np.testing.assert_allclose(b["states"], a["states"], atol=2e-5, rtol=0)
    np.testing.assert_allclose(b["z"], a["z"], atol=2e-5, rtol=0)
    check_grad(b["dp"], a["dp"], "c64", "dparams, prefix vs none")
    check_grad(b["di"], a["di"], "c64", "dinputs, prefix vs none")


# runs of consecutive diagonal ops (RZ, CZ) are merged into one factor per amplitude, and their backward
# gradients come from one pass (default with the Pauli frame): circuits dense in such runs, vs the oracle
def _diagonal_heavy_circuit(rng, n, g, n_params=6, n_inputs=2):
    """Runs of 2..8 diagonal ops (RZ on parameters and input columns, CZ), each followed by a few
    non-diagonal gates (H, RX, RY, CNOT) so that the phases the runs put in reach <Z> (a circuit of H
    layers and diagonal gates alone has <Z_i> = 0 and zero gradients for every angle)."""
    out = []
    while len(out) < g:
        for _ in range(int(rng.integers(2, 9))):
            if n >= 2 and rng.uniform() < 0.3:
                c, t = rng.choice(n, 2, replace=False)
                out.append(W.gate(W.CZ, (int(t),), (int(c),)))
            else:
                p = W.input_param(int(rng.integers(0, n_inputs))) if rng.uniform() < 0.3 else int(rng.integers(0, n_params))
                out.append(W.gate(W.RZ, (int(rng.integers(0, n)),), param=p))
        for _ in range(int(rng.integers(1, 4))):
            k = int(rng.choice([W.H, W.RX, W.RY, W.CNOT])) if n >= 2 else W.H
            if k == W.CNOT:
                c, t = rng.choice(n, 2, replace=False)
                out.append(W.gate(k, (int(t),), (int(c),)))
            elif k == W.H:
                out.append(W.gate(k, (int(rng.integers(0, n)),)))
            else:
                out.append(W.gate(k, (int(rng.integers(0, n)),), param=int(rng.integers(0, n_params))))
    return out + [W.gate(W.H, (qb,)) for qb in range(n)]


@pytest.mark.parametrize("seed,n,dtype,k,c,ckpt", [(60, 5, "c64", 4, 1, 0), (61, 8, "c128", 6, 2, 1),
                                                   (62, 11, "c64", 9, 3, 1), (63, 12, "c64", 12, 4, 0),
                                                   (64, 13, "c128", 11, 4, 0)])
def test_diagonal_runs_against_oracle(q, seed, n, dtype, k, c, ckpt):
    rng = np.random.default_rng(300 + seed)
    n_par, n_in, B = 6, 2, 3
    gates = [W.gate(W.H, (qb,)) for qb in range(n)] + _diagonal_heavy_circuit(rng, n, 10 * n, n_par, n_in)
    params = rng.uniform(0, 2 * math.pi, n_par)
    inputs = rng.uniform(0, math.pi, (B, n_in))
    g = rng.uniform(-1, 1, (B, n))
    wl = W.Workload("diag", n, B, dtype, gates, params, inputs, g)
    r = run(q, wl, dtype, "fused", k=k, contiguous_bits=c, checkpoint_passes=ckpt)
    assert "diagonal run" in r["plan"].kernel_source()
    pr, ir = rounded(wl, dtype)
    psi = oracle.simulate_strided(gates, n, pr, ir)
    t = TOL[dtype]
    np.testing.assert_allclose(r["states"], psi, atol=t["state"], rtol=0)
    np.testing.assert_allclose(r["z"], oracle.expval_z(psi, n), atol=t["z"], rtol=0)
    dp, di = oracle.grad_adjoint(gates, n, pr, ir, g)
    check_grad(r["dp"], dp, dtype, "dparams")
    check_grad(r["di"], di, dtype, "dinputs")


@pytest.mark.parametrize("which,dtype", [("c3", "c64"), ("hea", "c64"), ("hea", "c128")])
def test_merged_diagonal_runs_equal_split(q, which, dtype):
    wl = W.config(3, n=14, batch=4, dtype=dtype) if which == "c3" else W.Workload(
        "hea", 12, 3, dtype, W.hea_cz_ansatz(12, 4), *[np.random.default_rng(5).uniform(0, 3, s)
                                                       for s in ((96,), (3, 12), (3, 12))])
    k = 10 if dtype == "c64" else 9
    a = run(q, wl, dtype, "fused", k=k, checkpoint_passes=1, split_diagonal=True)
    b = run(q, wl, dtype, "fused", k=k, checkpoint_passes=1)
    t = 2e-5 if dtype == "c64" else 1e-12
    np.testing.assert_allclose(b["states"], a["states"], atol=t, rtol=0)
    np.testing.assert_allclose(b["z"], a["z"], atol=t, rtol=0)
    check_grad(b["dp"], a["dp"], dtype, "dparams, merged vs split")
    check_grad(b["di"], a["di"], dtype, "dinputs, merged vs split")


def test_pauli_frame_agrees_with_both_forms(q):
    # the same 14-qubit checkpointed workload both ways: results within the complex64 tolerances
    wl = W.config(3, n=14, batch=4)
    a = run(q, wl, "c64", "fused", k=10, checkpoint_passes=1, pauli_frame=False)
    b = run(q, wl, "c64", "fused", k=10, checkpoint_passes=1, pauli_frame=True)
    np.testing.assert_allclose(b["states"], a["states"], atol=2e-5, rtol=0)
    np.testing.assert_allclose(b["z"], a["z"], atol=2e-5, rtol=0)
    check_grad(b["dp"], a["dp"], "c64", "dparams, frame vs both forms")
    check_grad(b["di"], a["di"], "c64", "dinputs, frame vs both forms")


def _random_case(q, seed, n, dtype, mode, k, c, **kw):
    rng = np.random.default_rng(100 + seed)
    n_par, n_in, B = 7, 3, 3
    gates = random_circuit(rng, n, 8 * n + 10, n_par, n_in)
    params = rng.uniform(0, 2 * math.pi, n_par)
    inputs = rng.uniform(0, math.pi, (B, n_in))
    g = rng.uniform(-1, 1, (B, n))
    use_init = seed % 3 == 1
    init_np = None
    if use_init:
        init_np = rng.normal(size=(B, 2 ** n)) + 1j * rng.normal(size=(B, 2 ** n))
        init_np /= np.linalg.norm(init_np, axis=1, keepdims=True)
    wl = W.Workload("rand", n, B, dtype, gates, params, inputs, g)
    pr, ir = rounded(wl, dtype)
    cdt = torch.complex128 if dtype == "c128" else torch.complex64
    init = torch.tensor(init_np, dtype=cdt, device="cuda") if use_init else None
    r = run(q, wl, dtype, mode, init=init, k=k, contiguous_bits=c, **kw)
    init_ref = init.cpu().numpy().astype(np.complex128) if use_init else None
    psi = oracle.simulate_strided(gates, n, pr, ir, init=init_ref)
    t = TOL[dtype]
    np.testing.assert_allclose(r["states"], psi, atol=t["state"], rtol=0)
    np.testing.assert_allclose(r["z"], oracle.expval_z(psi, n), atol=t["z"], rtol=0)
    dp, di = oracle.grad_param_shift(gates, n, pr, ir, g, method="strided", init=init_ref)
    check_grad(r["dp"], dp, dtype, "dparams")
    check_grad(r["di"], di, dtype, "dinputs")


# ---------------------------------------------------------------- C2 (12 qubits, batch 1024, complex64)
@pytest.mark.parametrize("mode", ["fused", "per_gate"])
def test_c2_full_batch(q, mode):
    wl = W.config(2)
    r = run(q, wl, "c64", mode, backward=False)
    pr, ir = rounded(wl, "c64")
    zref = oracle.forward_z(wl.gates, wl.n, pr, ir[:32], method="strided")
    np.testing.assert_allclose(r["z"][:32], zref, atol=1e-5, rtol=0)
    norms = np.linalg.norm(r["states"], axis=1)
    np.testing.assert_allclose(norms, 1.0, atol=1e-5)


def test_c2_fused_equals_per_gate_all_samples(q):
    wl = W.config(2)
    a = run(q, wl, "c64", "fused", backward=False)
    b = run(q, wl, "c64", "per_gate", backward=False)
    np.testing.assert_allclose(a["z"], b["z"], atol=1e-5, rtol=0)
    np.testing.assert_allclose(a["states"], b["states"], atol=1e-5, rtol=0)


# ---------------------------------------------------------------- C3 (20 qubits, batch 64) at full size
_C3_REF = {}
C3_SAMPLES = 2          # samples carrying loss weight (their oracle states and gradients are computed)


def _c3_reference(wl, pr, ir, g):
    """FP64 oracle for samples 0, 1 of C3 (cached: the 20-qubit oracle is the slow part): Oracle-S
    states, every parameter and input gradient by the adjoint sweep, and the exact parameter shift on
    a seeded subset of 32 parameters and 4 input columns (parallel over the host's cores)."""
    if not _C3_REF:
        from oracle_pool import shift_derivatives
        S = C3_SAMPLES
        _C3_REF["psi"] = oracle.simulate_strided(wl.gates, wl.n, pr, ir[:S])
        _C3_REF["adj"] = oracle.grad_adjoint(wl.gates, wl.n, pr, ir[:S], g[:S])
        rng = np.random.default_rng(0x240409213)
        psub = sorted(rng.choice(wl.n_params, 32, replace=False).tolist())
        csub = sorted(rng.choice(wl.n_inputs, 4, replace=False).tolist())
        which = [i for i, gt in enumerate(wl.gates)
                 if (gt[3] >= 0 and gt[3] in psub) or (gt[3] <= -2 and -2 - gt[3] in csub)]
        d = shift_derivatives(wl.gates, wl.n, pr, ir[:S], g[:S], which)
        dps = {wl.gates[i][3]: v.sum() for i, v in d.items() if wl.gates[i][3] >= 0}
        dis = {-2 - wl.gates[i][3]: v for i, v in d.items() if wl.gates[i][3] <= -2}
        _C3_REF["shift"] = (psub, np.array([dps[p] for p in psub]), csub, np.stack([dis[c] for c in csub], axis=1))
    return _C3_REF["psi"], _C3_REF["adj"], _C3_REF["shift"]


def _elementwise_rel(got, ref, floor=0.05):
    """Worst per-element relative error over entries with |ref| >= floor * max|ref|."""
    got, ref = np.ravel(got), np.ravel(ref)
    m = np.abs(ref) >= floor * np.abs(ref).max()
    return float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m])))


# the bench's launch configuration: batch 64, checkpoint every pass, the tile sizes its autotuner picks
@pytest.mark.parametrize("k", [13, 12, 11])
def test_c3_full_size_against_oracle(q, k):
    wl = W.config(3)
    S = C3_SAMPLES
    # only samples 0 and 1 carry loss weight, so the batch-summed parameter gradient is checkable
    g = np.zeros_like(wl.grad_out)
    g[:S] = wl.grad_out[:S]
    wl.grad_out = g
    r = run(q, wl, "c64", "fused", k=k, checkpoint_passes=1)
    pr, ir = rounded(wl, "c64")
    norms = np.linalg.norm(r["states"], axis=1)
    np.testing.assert_allclose(norms, 1.0, atol=1e-5)
    psi, (adp, adi), (psub, sdp, csub, sdi) = _c3_reference(wl, pr, ir, g)
    np.testing.assert_allclose(r["states"][:S], psi, atol=1e-5, rtol=0)
    np.testing.assert_allclose(r["z"][:S], oracle.expval_z(psi, wl.n), atol=1e-5, rtol=0)
    # the oracle's two gradient methods agree (adjoint sweep vs exact shift rule)
    np.testing.assert_allclose(adp[psub], sdp, atol=1e-10 * np.abs(sdp).max())
    np.testing.assert_allclose(adi[:, csub], sdi, atol=1e-10 * np.abs(sdi).max())
    # all 400 parameter gradients and all 2 x 20 input gradients against the oracle, on the oracle's scale
    check_grad(r["dp"], adp, "c64", "C3 dparams (all 400)")
    for b in range(S):
        check_grad(r["di"][b], adi[b], "c64", f"C3 dinputs sample {b}")
    assert not np.any(r["di"][S:]), "samples without loss weight must get zero input gradients"
    # the seeded subset against the shift rule directly
    check_grad(r["dp"][psub], sdp, "c64", "C3 dparams, 32 by parameter shift")
    check_grad(r["di"][:S, csub], sdi, "c64", "C3 dinputs, 4 columns by parameter shift")
    # per element: every entry at least 5 % of the largest is within 1e-4 relative
    ep, ei = _elementwise_rel(r["dp"], adp), _elementwise_rel(r["di"][:S], adi)
    print(f"C3 k={k}: worst per-element relative gradient error dparams {ep:.2e} dinputs {ei:.2e}")
    assert ep <= 1e-4 and ei <= 1e-4, (ep, ei)


# ---------------------------------------------------------------- many tiles, every sample weighted
@pytest.mark.parametrize("k,ckpt", [(10, 1), (9, 0), (6, 1)])
def test_backward_many_tiles_all_samples(q, k, ckpt):
    """Far more tiles than resident CTAs (4096, 8192 and 65536) and every sample weighted, so every
    tile's gradient partials count: complex64 against the complex128 plan on every sample, and both
    against the FP64 oracle's adjoint sweep on the first and last sample. At k = 6 a tile has 2 threads
    (4 in complex128), so 16 (8) tiles share a CTA."""
    wl = W.ring_workload("many-tiles", 14, 256, 4, "c64", 7)
    r = run(q, wl, "c64", "fused", k=k, checkpoint_passes=ckpt)
    assert r["plan"].info()["n_passes"] >= 2
    pr, ir = rounded(wl, "c64")   # the complex128 plan takes the angles complex64 saw
    wl2 = W.Workload("many-tiles", wl.n, wl.batch, "c128", wl.gates, pr, ir, wl.grad_out)
    r2 = run(q, wl2, "c128", "fused", k=k, checkpoint_passes=ckpt)
    check_grad(r["dp"], r2["dp"], "c64", "dparams vs complex128")
    for b in (0, 1, 77, 128, 254, 255):
        check_grad(r["di"][b], r2["di"][b], "c64", f"dinputs sample {b} vs complex128")
    np.testing.assert_allclose(r["di"], r2["di"], atol=1e-4 * np.abs(r2["di"]).max())
    sel = [0, wl.batch - 1]
    adp, adi = oracle.grad_adjoint(wl.gates, wl.n, pr, ir[sel], wl.grad_out[sel])
    for j, b in enumerate(sel):
        check_grad(r["di"][b], adi[j], "c64", f"dinputs sample {b} vs oracle")
        check_grad(r2["di"][b], adi[j], "c128", f"complex128 dinputs sample {b} vs oracle")


# ---------------------------------------------------------------- backward vs central finite differences
@pytest.mark.parametrize("dtype,tol", [("c64", 1e-4), ("c128", 1e-7)])
def test_backward_against_central_finite_differences(q, dtype, tol):
    # the adjoint gradients against FP64 central differences of the oracle's loss (h = 1e-4: truncation
    # error ~1e-9 relative), on a multi-pass, checkpointed plan; inputs and parameters
    wl = W.config(3, n=10, batch=4, layers=3, dtype=dtype)
    r = run(q, wl, dtype, "fused", k=8, checkpoint_passes=1)
    assert r["plan"].info()["n_passes"] > 2
    pr, ir = rounded(wl, dtype)
    fp, fi = oracle.grad_finite_diff(wl.gates, wl.n, pr, ir, wl.grad_out, h=1e-4, method="strided")
    for got, ref, what in ((r["dp"], fp, "dparams"), (r["di"], fi, "dinputs")):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= tol, (what, rel)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max() + 1e-9, what


# ---------------------------------------------------------------- C5 ansatz at 12 qubits, checkpointed
@pytest.mark.parametrize("ckpt,rot", [(0, False), (1, False), (3, False), (0, True), (1, True), (2, True)])
def test_c5_ansatz_12q_checkpointed(q, ckpt, rot):
    # with rotating layouts the checkpoints hold states in the layouts the passes wrote
    wl = W.config(5, n=12, batch=2)
    r = run(q, wl, "c64", "fused", k=10 if rot else 8, checkpoint_passes=ckpt, rotate_low_bits=rot)
    if ckpt:
        assert r["plan"].info()["n_checkpoints"] >= 1
    pr, ir = rounded(wl, "c64")
    psi = oracle.simulate_strided(wl.gates, wl.n, pr, ir)
    np.testing.assert_allclose(r["z"], oracle.expval_z(psi, wl.n), atol=1e-5, rtol=0)
    subset = list(range(0, wl.n_params, 12))
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, pr, ir, wl.grad_out, method="strided",
                                     param_subset=subset)
    check_grad(r["dp"][subset], dp[subset], "c64", "C5@12q dparams subset")
    check_grad(r["di"], di, "c64", "C5@12q dinputs")


# ---------------------------------------------------------------- determinism, in-place init, edges
def test_bitwise_deterministic(q):
    wl = W.config(3, batch=4, layers=3)
    a = run(q, wl, "c64")
    b = run(q, wl, "c64")
    assert np.array_equal(a["z"], b["z"]) and np.array_equal(a["dp"], b["dp"]) and np.array_equal(a["di"], b["di"])


@pytest.mark.parametrize("frame", [False, True])
def test_inplace_init_and_empty_circuit(q, frame):
    n, B = 9, 2
    rng = np.random.default_rng(1)
    s = rng.normal(size=(B, 2 ** n)) + 1j * rng.normal(size=(B, 2 ** n))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    st = torch.tensor(s, dtype=torch.complex64, device="cuda")
    plan = q.Plan([], n, pauli_frame=frame)
    out, z = plan.forward(None, None, init=st, states=st)
    torch.cuda.synchronize()
    np.testing.assert_allclose(z.cpu().numpy(), oracle.expval_z(st.cpu().numpy().astype(complex), n), atol=1e-6)
    np.testing.assert_allclose(out.cpu().numpy(), s.astype(np.complex64), atol=1e-6)
    wl = W.config(3, n=n, batch=B, layers=2)
    plan = q.Plan(wl.gates, n, k=6, pauli_frame=frame)
    p, x, g = tensors(wl, "c64")
    st2 = torch.tensor(s, dtype=torch.complex64, device="cuda")
    out, z = plan.forward(p, x, init=st2, states=st2)
    pr, ir = rounded(wl, "c64")
    psi = oracle.simulate_strided(wl.gates, n, pr, ir, init=s.astype(np.complex64).astype(complex))
    np.testing.assert_allclose(out.cpu().numpy(), psi, atol=1e-5)


def test_expval_z_standalone(q):
    rng = np.random.default_rng(4)
    for n, B, dt in ((1, 3, torch.complex64), (5, 2, torch.complex128), (13, 3, torch.complex64),
                     (16, 2, torch.complex128)):
        s = rng.normal(size=(B, 2 ** n)) + 1j * rng.normal(size=(B, 2 ** n))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        st = torch.tensor(s, dtype=dt, device="cuda")
        z = q.expval_z(st, n).cpu().numpy()
        np.testing.assert_allclose(z, oracle.expval_z(st.cpu().numpy().astype(complex), n),
                                   atol=1e-6 if dt == torch.complex64 else 1e-13)


def test_autograd_layer(q):
    wl = W.config(3, n=8, batch=4, layers=3)
    layer = q.QSimLayer(wl.gates, wl.n, init_params=wl.params).cuda()
    x = torch.tensor(wl.inputs, dtype=torch.float32, device="cuda", requires_grad=True)
    z = layer(x)
    loss = (torch.tensor(wl.grad_out, device="cuda") * z).sum()
    loss.backward()
    pr, ir = rounded(wl, "c64")
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, pr, ir, wl.grad_out, method="strided")
    check_grad(layer.weight.grad.double().cpu().numpy(), dp, "c64", "layer dparams")
    check_grad(x.grad.double().cpu().numpy(), di, "c64", "layer dinputs")
