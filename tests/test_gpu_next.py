"""Strongly Entangling Layers with data re-uploading, OpenQASM programs and gradient landscapes on the
GPU path, against the FP64 oracle."""
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


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_sel_reuploading_against_oracle(q, dtype):
    # the inputs enter before every layer: dL/dinputs sums the occurrences of each column
    wl = W.sel_workload("sel", 6, 3, 3, dtype, seed=31, reupload=True)
    p, x, g = tensors(wl, dtype)
    plan = q.Plan(wl.gates, wl.n, dtype=dtype, k=4, contiguous_bits=2)
    states, z = plan.forward(p, x)
    dp, di = plan.backward(g)
    torch.cuda.synchronize()
    pr, xr = rounded(wl, dtype)
    psi = oracle.simulate_kron(wl.gates, wl.n, pr, xr)
    t = TOL[dtype]
    np.testing.assert_allclose(states.cpu().numpy(), psi, atol=t["state"], rtol=0)
    np.testing.assert_allclose(z.cpu().numpy(), oracle.expval_z(psi, wl.n), atol=t["z"], rtol=0)
    rdp, rdi = oracle.grad_param_shift(wl.gates, wl.n, pr, xr, wl.grad_out)
    check_grad(dp.cpu().numpy(), rdp, dtype, "SEL dparams")
    check_grad(di.cpu().numpy(), rdi, dtype, "SEL dinputs")


def test_sel_long_range_cnots_several_passes(q):
    # ranges r = 1..n-1 make CNOTs between distant qubits; k = 8 of 12 forces several passes
    wl = W.sel_workload("sel12", 12, 2, 4, "c64", seed=32, reupload=True)
    p, x, g = tensors(wl, "c64")
    plan = q.Plan(wl.gates, wl.n, k=8)
    assert plan.info()["n_passes"] > 2
    _, z = plan.forward(p, x)
    dp, di = plan.backward(g)
    torch.cuda.synchronize()
    pr, xr = rounded(wl, "c64")
    psi = oracle.simulate_strided(wl.gates, wl.n, pr, xr)
    np.testing.assert_allclose(z.cpu().numpy(), oracle.expval_z(psi, wl.n), atol=TOL["c64"]["z"], rtol=0)
    subset = list(range(0, wl.n_params, 7))
    rdp, rdi = oracle.grad_param_shift(wl.gates, wl.n, pr, xr, wl.grad_out, method="strided", param_subset=subset)
    check_grad(dp.cpu().numpy()[subset], rdp[subset], "c64", "SEL12 dparams subset")
    check_grad(di.cpu().numpy(), rdi, "c64", "SEL12 dinputs")


def test_qasm_program_runs_on_the_gpu(q):
    text = """OPENQASM 2.0;
include "qelib1.inc";
qreg a[2]; qreg b[3];
h a[0];
cx a[0], a[1];
cx a[1], b;
ry(pi/3) b[2];
rz(-0.7) a;
rx(2*pi/5) b[0];
cz b[1], a[0];
"""
    gates, params, n = q.parse_qasm(text)
    plan = q.Plan(gates, n, dtype="c128")
    states, z = plan.forward(torch.tensor(params, dtype=torch.float64, device="cuda"),
                             torch.zeros((1, 0), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    psi = oracle.simulate_kron(gates, n, params, np.zeros((1, 0)))
    np.testing.assert_allclose(states.cpu().numpy(), psi, atol=1e-12, rtol=0)
    np.testing.assert_allclose(z.cpu().numpy(), oracle.expval_z(psi, n), atol=1e-12, rtol=0)


@pytest.mark.parametrize("remap", [False, True])
def test_gradient_landscape_against_oracle(q, remap):
    n, layers = 3, 2
    gates = W.sel_ansatz(n, layers, encode=False)
    P = W.count_params(gates)
    rng = np.random.default_rng(5)
    base = rng.uniform(-math.pi, math.pi, P)
    values = np.linspace(-math.pi, math.pi, 7)
    weights = rng.uniform(-1, 1, n)
    grid, z = q.landscape(gates, n, torch.tensor(base, device="cuda", dtype=torch.float64),
                          torch.tensor(values, device="cuda", dtype=torch.float64),
                          torch.tensor(weights, device="cuda"), dtype="c128", weight_remap=remap, z=True)
    torch.cuda.synchronize()
    grid, z = grid.cpu().numpy(), z.cpu().numpy()
    assert grid.shape == (P, len(values))
    none = np.zeros((1, 0))
    for k in range(P):
        for v, val in enumerate(values):
            th = base.copy()
            th[k] = val
            if remap:
                dp, _ = oracle.grad_remapped(gates, n, th, none, weights[None], param_subset=[k])
                zr = oracle.forward_z_remapped(gates, n, th, none)
            else:
                dp, _ = oracle.grad_param_shift(gates, n, th, none, weights[None], param_subset=[k])
                zr = oracle.forward_z(gates, n, th, none)
            assert abs(grid[k, v] - dp[k]) <= 1e-11, (k, v, grid[k, v], dp[k])
            np.testing.assert_allclose(z[k * len(values) + v], zr[0], atol=1e-12)


def test_gradient_landscape_single_precision_and_errors(q):
    gates = W.sel_ansatz(4, 1, encode=False)
    P = W.count_params(gates)
    base = torch.zeros(P, device="cuda")
    values = torch.linspace(-1.0, 1.0, 4, device="cuda")
    grid = q.landscape(gates, 4, base, values, torch.ones(4, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.isfinite(grid).all() and grid.shape == (P, 4)
    with pytest.raises(q.QsimError):
        q.landscape(W.sel_ansatz(4, 1, encode=True), 4, base, values, torch.ones(4, dtype=torch.float64, device="cuda"))


def test_gradient_landscape_repeated_calls_reuse_the_plan(q):
    # the same circuit swept three times (the plan and buffers are kept), once on a side stream
    n = 3
    gates = W.sel_ansatz(n, 2, encode=False)
    P = W.count_params(gates)
    rng = np.random.default_rng(8)
    weights = rng.uniform(-1, 1, n)
    values = np.linspace(-3.0, 3.0, 5)
    side = torch.cuda.Stream()
    none = np.zeros((1, 0))
    for it in range(3):
        base = rng.uniform(-math.pi, math.pi, P)
        args = (gates, n, torch.tensor(base, device="cuda", dtype=torch.float64),
                torch.tensor(values, device="cuda", dtype=torch.float64), torch.tensor(weights, device="cuda"))
        grid = q.landscape(*args, dtype="c128", stream=side if it == 1 else None)
        torch.cuda.synchronize()
        grid = grid.cpu().numpy()
        for kk in (0, P // 2, P - 1):
            for v in (0, 4):
                th = base.copy()
                th[kk] = values[v]
                dp, _ = oracle.grad_param_shift(gates, n, th, none, weights[None], param_subset=[kk])
                assert abs(grid[kk, v] - dp[kk]) <= 1e-11, (it, kk, v)
    q.landscape_clear_cache()
