"""Deep circuits on few qubits against the FP64 oracle. Inside a fused pass rotations and Hadamards run
unnormalised (a tangent or cotangent coefficient, the cos / sin factored out and applied later), so
each one may grow the tile's values by up to sqrt(2); the planner adds a rescale op after every 48 of
them and caps a pass at 256. The angles here sit near the largest growth: without rescaling, the
backward's lambda-psi products of a 256-rotation pass would leave the complex64 range (2^128)."""
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


def worst_case(name, n, layers, batch, dtype, seed, hadamards=0):
    wl = W.ring_workload(name, n, batch, layers, dtype, seed)
    wl.gates = wl.gates + [W.gate(W.H, (i % n,)) for i in range(hadamards)]
    # angles within 0.4 of pi/2 or 3 pi/2, where the half angle's tangent is near +-1: ~0.37 bits of
    # growth per rotation, 190 bits for the backward's products over a 256-rotation pass (exactly
    # pi/2 would make the circuit Clifford, with gradients near zero)
    rng = np.random.default_rng(seed)
    band = lambda a: math.pi / 2 + math.pi * rng.integers(0, 2, a.shape) + rng.uniform(-0.4, 0.4, a.shape)
    wl.params = band(wl.params)
    wl.inputs = band(wl.inputs)
    return wl


@pytest.mark.parametrize("dtype,frame", [("c64", False), ("c128", False), ("c64", True)])
def test_deep_circuit_worst_case_growth(q, dtype, frame):
    wl = worst_case("deep8", 8, 32, 3, dtype, seed=41, hadamards=40)   # 520 rotations + 40 H on 8 qubits
    p, x, g = tensors(wl, dtype)
    plan = q.Plan(wl.gates, wl.n, dtype=dtype, pauli_frame=frame)
    d = plan.describe()
    assert len(d["passes"]) >= 3
    assert any(op["kind"] == "scale" for ps in d["passes"] for ph in ps["phases"] for op in ph["ops"])
    states, z = plan.forward(p, x)
    dp, di = plan.backward(g)
    torch.cuda.synchronize()
    pr, xr = rounded(wl, dtype)
    psi = oracle.simulate_strided(wl.gates, wl.n, pr, xr)
    t = TOL[dtype]
    np.testing.assert_allclose(states.cpu().numpy(), psi, atol=t["state"], rtol=0)
    np.testing.assert_allclose(z.cpu().numpy(), oracle.expval_z(psi, wl.n), atol=t["z"], rtol=0)
    subset = list(range(0, wl.n_params, 23)) + [wl.n_params - 1]
    rdp, rdi = oracle.grad_param_shift(wl.gates, wl.n, pr, xr, wl.grad_out, method="strided", param_subset=subset)
    check_grad(dp.cpu().numpy()[subset], rdp[subset], dtype, "deep dparams subset")
    check_grad(di.cpu().numpy(), rdi, dtype, "deep dinputs")


def test_deep_circuit_in_the_multi_circuit_queue(q):
    # the same range control inside the persistent multi-circuit kernels (one deep circuit among small ones)
    wls = [worst_case("deep6", 6, 24, 2, "c64", seed=43),
           W.ring_workload("small4", 4, 2, 2, "c64", seed=44)]
    B = 2
    mp = q.MultiPlan([(w.gates, w.n) for w in wls])
    p = torch.tensor(np.concatenate([w.params for w in wls]), dtype=torch.float32, device="cuda")
    x = torch.tensor(np.concatenate([w.inputs.ravel() for w in wls]), dtype=torch.float32, device="cuda")
    g = torch.tensor(np.concatenate([w.grad_out.ravel() for w in wls]), dtype=torch.float64, device="cuda")
    _, z = mp.forward(p, x, B)
    dp, di = mp.backward(g)
    torch.cuda.synchronize()
    assert mp.sync_status() == 0
    off = mp.offsets(B)
    for c, w in enumerate(wls):
        pr, xr = rounded(w, "c64")
        psi = oracle.simulate_strided(w.gates, w.n, pr, xr)
        zc = z[int(off["z"][c]):int(off["z"][c + 1])].cpu().numpy().reshape(B, w.n)
        np.testing.assert_allclose(zc, oracle.expval_z(psi, w.n), atol=TOL["c64"]["z"], rtol=0)
        subset = list(range(0, w.n_params, 17))
        rdp, rdi = oracle.grad_param_shift(w.gates, w.n, pr, xr, w.grad_out, method="strided", param_subset=subset)
        dpc = dp[int(off["params"][c]):int(off["params"][c + 1])].cpu().numpy()
        check_grad(dpc[subset], rdp[subset], "c64", f"circuit {c} dparams subset")
        dic = di[int(off["inputs"][c]):int(off["inputs"][c + 1])].cpu().numpy().reshape(B, w.n_inputs)
        check_grad(dic, rdi, "c64", f"circuit {c} dinputs")
