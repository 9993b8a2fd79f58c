"""Several circuits of uneven size in one persistent launch per direction (work queue), against the
FP64 oracle and against the single-circuit path; CUDA-graph replay; the bounded-wait timeout."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_util import check_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def concat(wls, B, dtype):
    rd = torch.float64 if dtype == "c128" else torch.float32
    p = torch.tensor(np.concatenate([w.params for w in wls]), dtype=rd, device="cuda")
    x = torch.tensor(np.concatenate([w.inputs[:B].ravel() for w in wls]), dtype=rd, device="cuda")
    g = torch.tensor(np.concatenate([w.grad_out[:B].ravel() for w in wls]), dtype=torch.float64, device="cuda")
    return p, x, g


def split(t, off, c):
    return t[int(off[c]):int(off[c + 1])]


def run_multi(q, wls, B, dtype="c64", graph=False, reps=1, **kw):
    mp = q.MultiPlan([(w.gates, w.n) for w in wls], dtype=dtype, graph=graph, **kw)
    p, x, g = concat(wls, B, dtype)
    outs = []
    for _ in range(reps):
        states, z = mp.forward(p, x, B)
        dp, di = mp.backward(g)
        torch.cuda.synchronize()
        assert mp.sync_status() == 0
        outs.append((states.clone(), z.clone(), dp.clone(), di.clone()))
    return mp, outs


def small_set(n_circ=10, seed=11):
    return W.multi_circuit_config(n_circuits=n_circ, n_min=3, n_max=14, d_min=1, d_max=3, seed=seed)


# large: circuits of at least this many qubits run as their own single-circuit plans (-1: none), so
# the same launch mixes queue circuits and own-plan circuits on one set of buffers
@pytest.mark.parametrize("dtype,large", [("c64", -1), ("c128", -1), ("c64", 9), ("c128", 12)])
def test_multi_against_oracle(q, dtype, large):
    wls = small_set()
    B = 4
    mp, [(states, z, dp, di)] = run_multi(q, wls, B, dtype, large_qubits=large)
    off = mp.offsets(B)
    tol = 1e-5 if dtype == "c64" else 1e-12
    for c, w in enumerate(wls):
        pr = w.params.astype(np.float32).astype(float) if dtype == "c64" else w.params
        ir = w.inputs.astype(np.float32).astype(float) if dtype == "c64" else w.inputs
        psi = oracle.simulate_strided(w.gates, w.n, pr, ir)
        zc = split(z, off["z"], c).cpu().numpy().reshape(B, w.n)
        np.testing.assert_allclose(zc, oracle.expval_z(psi, w.n), atol=tol, rtol=0)
        sc = split(states, off["states"], c).cpu().numpy().reshape(B, 2 ** w.n)
        np.testing.assert_allclose(sc, psi, atol=tol, rtol=0)
        rp, ri = oracle.grad_param_shift(w.gates, w.n, pr, ir, w.grad_out, method="strided")
        check_grad(split(dp, off["params"], c).cpu().numpy(), rp, dtype, f"circuit {c} dparams")
        check_grad(split(di, off["inputs"], c).cpu().numpy().reshape(B, w.n_inputs), ri, dtype, f"circuit {c} dinputs")


def test_c4_full_against_single_circuit_path(q):
    wls = W.multi_circuit_config()            # 256 circuits, 8..22 qubits, batch 4
    B = 4
    mp, [(states, z, dp, di)] = run_multi(q, wls, B)
    off = mp.offsets(B)
    inf = mp.info()
    assert inf["n_circuits"] == 256 and inf["items_fwd"] > 256
    rng = np.random.default_rng(0)
    check = sorted(set(rng.choice(256, 24, replace=False).tolist()) | {int(np.argmax([w.n for w in wls]))})
    for c in check:
        w = wls[c]
        plan = q.Plan(w.gates, w.n)
        p = torch.tensor(w.params, dtype=torch.float32, device="cuda")
        x = torch.tensor(w.inputs, dtype=torch.float32, device="cuda")
        _, zs = plan.forward(p, x)
        dps, dis = plan.backward(torch.tensor(w.grad_out, dtype=torch.float64, device="cuda"))
        np.testing.assert_allclose(split(z, off["z"], c).cpu().numpy().reshape(B, w.n), zs.cpu().numpy(), atol=1e-6)
        check_grad(split(dp, off["params"], c).cpu().numpy(), dps.cpu().numpy(), "c64", f"C4[{c}] dparams")
        check_grad(split(di, off["inputs"], c).cpu().numpy(), dis.cpu().numpy().ravel(), "c64", f"C4[{c}] dinputs")
        del plan
    # oracle on the smaller circuits of the set
    for c in [i for i in check if wls[i].n <= 12][:6]:
        w = wls[c]
        pr, ir = w.params.astype(np.float32).astype(float), w.inputs.astype(np.float32).astype(float)
        zr = oracle.forward_z(w.gates, w.n, pr, ir, method="strided")
        np.testing.assert_allclose(split(z, off["z"], c).cpu().numpy().reshape(B, w.n), zr, atol=1e-5)


def test_c4_full_against_oracle_above_12_qubits(q):
    # the whole 256-circuit launch, with the FP64 oracle on sample 0 of three circuits above 12 qubits:
    # the first 22-qubit circuit of the set, the shortest 22-qubit one and the first between 15 and 18
    # qubits. Their other samples carry no loss weight, so the circuit's batch-summed parameter gradient
    # is sample 0's alone.
    from oracle_pool import shift_derivatives
    wls = W.multi_circuit_config()
    B = 4
    big = [i for i, w in enumerate(wls) if w.n == 22]
    check = [big[0], min(big, key=lambda i: len(wls[i].gates)),
             next(i for i, w in enumerate(wls) if 15 <= w.n <= 18)]
    for c in check:
        wls[c].grad_out = np.array(wls[c].grad_out, copy=True)
        wls[c].grad_out[1:] = 0.0
    mp, [(states, z, dp, di)] = run_multi(q, wls, B)
    off = mp.offsets(B)
    for c in check:
        w = wls[c]
        pr, ir = w.params.astype(np.float32).astype(float), w.inputs.astype(np.float32).astype(float)
        psi = oracle.simulate_strided(w.gates, w.n, pr, ir[:1])
        zc = split(z, off["z"], c).cpu().numpy().reshape(B, w.n)
        np.testing.assert_allclose(zc[:1], oracle.expval_z(psi, w.n), atol=1e-5, rtol=0)
        sc = split(states, off["states"], c).cpu().numpy().reshape(B, 2 ** w.n)
        np.testing.assert_allclose(sc[:1], psi, atol=1e-5, rtol=0)
        adp, adi = oracle.grad_adjoint(w.gates, w.n, pr, ir[:1], w.grad_out[:1])
        gdp = split(dp, off["params"], c).cpu().numpy()
        gdi = split(di, off["inputs"], c).cpu().numpy().reshape(B, w.n_inputs)
        check_grad(gdp, adp, "c64", f"C4[{c}] ({w.n} qubits) dparams, sample 0")
        check_grad(gdi[0], adi[0], "c64", f"C4[{c}] ({w.n} qubits) dinputs, sample 0")
        assert not np.any(gdi[1:]), "samples without loss weight must get zero input gradients"
        # a few entries by the exact shift rule: two parameters of the last layer and one input column
        rot = [i for i, gt in enumerate(w.gates) if gt[3] >= 0]
        enc = [i for i, gt in enumerate(w.gates) if gt[3] <= -2]
        d = shift_derivatives(w.gates, w.n, pr, ir[:1], w.grad_out[:1], [rot[-1], rot[-2], enc[w.n // 2]])
        for i, v in d.items():
            ref = v[0]
            got = gdp[w.gates[i][3]] if w.gates[i][3] >= 0 else gdi[0, -2 - w.gates[i][3]]
            assert abs(got - ref) <= 1e-4 * np.abs(adp).max() + 1e-7, (c, i, got, ref)


@pytest.mark.parametrize("large", [-1, 8])
def test_multi_graph_replay_is_identical(q, large):
    wls = small_set(6, seed=3)
    mp, outs = run_multi(q, wls, 4, graph=True, reps=3, large_qubits=large)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_multi_bounded_wait_reports_timeout(q):
    # the first circuit has several passes, so items of its second pass wait on its first pass;
    # withholding item 0's completion makes those waits run out after 20 ms
    wls = [W.Workload("big", 16, 2, "c64", W.hea_cz_ansatz(16, 2), np.zeros(64), np.zeros((2, 16)),
                      np.ones((2, 16)))] + small_set(3, seed=5)
    mp = q.MultiPlan([(w.gates, w.n) for w in wls])
    p, x, g = concat(wls, 2, "c64")
    mp.set_test_hooks(withhold_item=0, timeout_ns=20_000_000)
    mp.forward(p, x, 2)
    torch.cuda.synchronize()
    assert mp.sync_status() == -8
    mp.set_test_hooks(withhold_item=-1, timeout_ns=0)
    _, z = mp.forward(p, x, 2)
    torch.cuda.synchronize()
    assert mp.sync_status() == 0
    zb = z[:32].cpu().numpy()
    assert np.all(np.isfinite(zb)) and abs(zb.reshape(2, 16)[0, 0] - 1.0) < 1e-5   # RY/RZ(0) circuit keeps |0>
