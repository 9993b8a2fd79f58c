"""Quantum weight remapping (angle = pi * tanh(weight) for trainable weights, Sec. "Additional Optimizations") on the GPU
path against the FP64 oracle: states, <Z> and dL/dweights through the chain rule, single and
multi-circuit plans, fused and per-gate modes."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_util import TOL, check_grad, rounded, tensors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def weights(wl):
    w = wl.params - math.pi      # both signs, some large enough to saturate tanh
    w[::5] *= 2.0
    return w


@pytest.mark.parametrize("dtype,mode", [("c128", "fused"), ("c64", "fused"), ("c64", "per_gate")])
def test_remap_against_oracle(q, dtype, mode):
    wl = W.config(1, n=5, batch=3, layers=2, dtype=dtype)
    wl.params = weights(wl)
    p, x, g = tensors(wl, dtype)
    kw = dict(k=3, contiguous_bits=1) if mode == "fused" else {}
    plan = q.Plan(wl.gates, wl.n, dtype=dtype, mode=mode, weight_remap=True, **kw)
    states, z = plan.forward(p, x)
    dp, di = plan.backward(g)
    torch.cuda.synchronize()
    pr, xr = rounded(wl, dtype)
    psi = oracle.simulate_kron(wl.gates, wl.n, oracle.remap(pr), xr)
    t = TOL[dtype]
    assert np.abs(states.cpu().numpy() - psi).max() <= t["state"]
    assert np.abs(z.cpu().numpy() - oracle.expval_z(psi, wl.n)).max() <= t["z"]
    rdp, rdi = oracle.grad_remapped(wl.gates, wl.n, pr, xr, wl.grad_out)
    check_grad(dp.cpu().numpy(), rdp, dtype, "dweights")
    check_grad(di.cpu().numpy(), rdi, dtype, "dinputs")


def test_remapped_weights_that_map_onto_the_plain_angles(q):
    # weights atanh(a / pi) remap to the angles a: the remapped plan must reproduce the plain one
    wl = W.config(1, n=4, batch=2, layers=2, dtype="c128")
    p, x, g = tensors(wl)
    a = torch.remainder(p + math.pi, 2 * math.pi) - math.pi       # the same rotations, angles in [-pi, pi)
    a = a.clamp(-0.999 * math.pi, 0.999 * math.pi)
    plain = q.Plan(wl.gates, wl.n, dtype="c128")
    remapped = q.Plan(wl.gates, wl.n, dtype="c128", weight_remap=True)
    z0 = plain.forward(a, x)[1]
    z1 = remapped.forward(torch.atanh(a / math.pi), x)[1]
    torch.cuda.synchronize()
    assert np.abs((z1 - z0).cpu().numpy()).max() <= 1e-12


def test_remap_multi_circuit(q):
    wls = W.multi_circuit_config(n_circuits=4, n_min=3, n_max=9, d_min=1, d_max=2, seed=17)
    B = 2
    for w in wls:
        w.params = weights(w)
    mp = q.MultiPlan([(w.gates, w.n) for w in wls], weight_remap=True)
    p = torch.tensor(np.concatenate([w.params for w in wls]), dtype=torch.float32, device="cuda")
    x = torch.tensor(np.concatenate([w.inputs[:B].ravel() for w in wls]), dtype=torch.float32, device="cuda")
    g = torch.tensor(np.concatenate([w.grad_out[:B].ravel() for w in wls]), dtype=torch.float64, device="cuda")
    _, z = mp.forward(p, x, B)
    dp, di = mp.backward(g)
    torch.cuda.synchronize()
    assert mp.sync_status() == 0
    off = mp.offsets(B)
    for c, w in enumerate(wls):
        pr, xr = rounded(w, "c64")
        xr = xr[:B]
        zc = z[int(off["z"][c]):int(off["z"][c + 1])].cpu().numpy().reshape(B, w.n)
        np.testing.assert_allclose(zc, oracle.forward_z_remapped(w.gates, w.n, pr, xr), atol=TOL["c64"]["z"])
        rdp, rdi = oracle.grad_remapped(w.gates, w.n, pr, xr, w.grad_out[:B])
        check_grad(dp[int(off["params"][c]):int(off["params"][c + 1])].cpu().numpy(), rdp, "c64", f"dweights[{c}]")
        check_grad(di[int(off["inputs"][c]):int(off["inputs"][c + 1])].cpu().numpy(), rdi.ravel(), "c64", f"dinputs[{c}]")
