"""30 qubits, batch 1 (8 GiB complex64 state), forward + checkpointed adjoint backward.

No oracle can hold this state, so the full-size run is pinned by facts that hold at any size
(the 12-qubit version of the same ansatz is compared with the oracle in test_gpu_parity.py):
product-state closed forms for <Z> and gradients, the CNOT ring on basis states (exact +-1, a
bit-exact check of every pass's index maps at this size), the forward followed by its inverse
returning |0...0>, norm preservation, agreement of complex64 with the complex128 GPU mode, and
checkpointed vs non-checkpointed gradients.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import check_grad

pytestmark = pytest.mark.gpu
N = 30


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def _run(q, gates, params, inputs, g, dtype="c64", **kw):
    rd = torch.float64 if dtype == "c128" else torch.float32
    plan = q.Plan(gates, N, dtype=dtype, **kw)
    p = torch.tensor(params, dtype=rd, device="cuda")
    x = torch.tensor(inputs, dtype=rd, device="cuda")
    states, z = plan.forward(p, x)
    out = {"z": z.cpu().numpy(), "norm": float(states.abs().pow(2).sum().item())}
    if g is not None:
        dp, di = plan.backward(torch.tensor(g, dtype=torch.float64, device="cuda"))
        out["dp"], out["di"] = dp.cpu().numpy(), di.cpu().numpy()
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    out["info"] = plan.info()
    del plan, states
    torch.cuda.empty_cache()
    return out


def test_product_state_closed_forms_30q(q):
    rng = np.random.default_rng(30)
    x = rng.uniform(0, math.pi, (1, N))
    y = rng.uniform(0, 2 * math.pi, N)
    gates = [W.gate(W.RX, (k,), param=W.input_param(k)) for k in range(N)]
    gates += [W.gate(W.RY, (k,), param=k) for k in range(N)]
    g = rng.uniform(-1, 1, (1, N))
    r = _run(q, gates, y, x, g, checkpoint_passes=1)
    xf, yf = x.astype(np.float32).astype(float), y.astype(np.float32).astype(float)
    np.testing.assert_allclose(r["z"], np.cos(xf) * np.cos(yf)[None], atol=1e-5)
    check_grad(r["dp"], np.sum(-g * np.cos(xf) * np.sin(yf)[None], axis=0), "c64", "30q product dparams")
    check_grad(r["di"], -g * np.sin(xf) * np.cos(yf)[None], "c64", "30q product dinputs")
    assert abs(r["norm"] - 1.0) < 1e-5


def test_cnot_ring_basis_state_30q(q):
    bits = [(k * 7 + 3) % 2 for k in range(N)]
    gates = [W.gate(W.X, (k,)) for k in range(N) if bits[k]]
    for _ in range(3):
        gates += [W.gate(W.CNOT, ((k + 1) % N,), (k,)) for k in range(N)]
    b = list(bits)
    for _ in range(3):
        for k in range(N):
            b[(k + 1) % N] ^= b[k]
    r = _run(q, gates, np.zeros(0), np.zeros((1, 0)), None)
    np.testing.assert_array_equal(r["z"][0], [1.0 - 2.0 * v for v in b])


def test_forward_then_inverse_is_identity_30q(q):
    wl = W.config(5, layers=2)
    inv = []
    for gt in reversed(wl.gates):
        if gt[0] in (W.RX, W.RY, W.RZ):
            inv.append(gt)            # inverse angle through negated parameter copies below
        else:
            inv.append(gt)
    P = wl.n_params
    n_in = wl.n_inputs
    # second half uses negated angles: params [p, -p], inputs [x, -x]
    gates = list(wl.gates)
    for gt in inv:
        k, t, c, p = gt
        if p >= 0:
            gates.append((k, t, c, p + P))
        elif p <= -2:
            gates.append((k, t, c, -2 - ((-2 - p) + n_in)))
        else:
            gates.append(gt)
    params = np.concatenate([wl.params, -wl.params])
    inputs = np.concatenate([wl.inputs, -wl.inputs], axis=1)
    r = _run(q, gates, params, inputs, None)
    np.testing.assert_allclose(r["z"][0], np.ones(N), atol=2e-5)   # |0...0> has <Z_i> = 1


def test_c5_complex64_vs_complex128_and_checkpoints(q):
    wl = W.config(5)
    a = _run(q, wl.gates, wl.params, wl.inputs, wl.grad_out, "c64", checkpoint_passes=8)
    assert a["info"]["n_checkpoints"] >= 2
    assert abs(a["norm"] - 1.0) < 1e-4
    b = _run(q, wl.gates, wl.params, wl.inputs, wl.grad_out, "c128", checkpoint_passes=8)
    np.testing.assert_allclose(a["z"], b["z"], atol=1e-5)
    check_grad(a["dp"], b["dp"], "c64", "C5 dparams c64 vs c128")
    check_grad(a["di"], b["di"], "c64", "C5 dinputs c64 vs c128")
    c = _run(q, wl.gates, wl.params, wl.inputs, wl.grad_out, "c64", checkpoint_passes=0)
    np.testing.assert_allclose(a["z"], c["z"], atol=0)
    check_grad(a["dp"], c["dp"], "c64", "C5 checkpointed vs not")
