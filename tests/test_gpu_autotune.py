"""Tile-size autotuner: candidates timed on the device, the winner is a valid k, and plans built with
autotuned per-circuit k values give the same results as the default plans (the oracle pins those)."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import TOL, check_grad, tensors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def test_autotune_times_three_candidates(q):
    wl = W.config(3, n=15, batch=4, layers=3)
    k, ms = q.autotune(wl.gates, wl.n, 4, reps=1)
    assert k in (11, 12, 13)
    assert ms[3] == -1.0   # three tile sizes; the fourth slot is for single-pass circuits
    ms = ms[:3]
    assert all(m > 0 for m in ms)
    # the largest k within 2 % of the fastest candidate
    assert ms[k - 11] <= 1.02 * min(ms)
    assert all(m > 1.02 * min(ms) for m in ms[k - 11 + 1:])


def test_autotune_single_pass_when_the_state_fits(q):
    # one pass holds the whole state: k = n, and the four candidates are 2^5 and 2^4 amplitudes per
    # thread with the Pauli frame and without it; the fastest wins, and the tuned plan gives the default
    # plan's results
    wl = W.config(2, batch=8)
    k, ms, tuned = q.autotune(wl.gates, wl.n, 8, reps=1, return_opts=True)
    assert k == wl.n and all(m > 0 for m in ms)
    best = int(np.argmin(ms))
    assert tuned["fwd_reg_bits"] == (0 if best in (0, 2) else 4) and tuned["bwd_reg_bits"] == tuned["fwd_reg_bits"]
    assert tuned["pauli_frame"] == (best in (0, 1))
    p, x, g = tensors(wl)
    a = q.Plan(wl.gates, wl.n)
    b = q.Plan(wl.gates, wl.n, **tuned)
    for fr, frame in ((4, True), (5, False), (4, False)):   # every candidate, not only the one that won
        c = q.Plan(wl.gates, wl.n, fwd_reg_bits=fr, bwd_reg_bits=fr, pauli_frame=frame)
        _, zc = c.forward(p, x)
        _, za = a.forward(p, x)
        torch.cuda.synchronize()
        np.testing.assert_allclose(zc.cpu().numpy(), za.cpu().numpy(), atol=1e-5)
        np.testing.assert_allclose(c.backward(g)[0].cpu().numpy(), a.backward(g)[0].cpu().numpy(), atol=1e-4)
    _, zb = b.forward(p, x)
    torch.cuda.synchronize()
    np.testing.assert_allclose(zb.cpu().numpy(), a.forward(p, x)[1].cpu().numpy(), atol=1e-5)
    # an explicit register choice is kept: nothing is timed
    k2, ms2 = q.autotune(wl.gates, wl.n, 8, fwd_reg_bits=4)
    assert k2 == wl.n and ms2 == [-1.0, -1.0, -1.0, -1.0]


def test_autotuned_plan_matches_default_plan(q):
    wl = W.config(3, n=14, batch=4, layers=2)
    p, x, g = tensors(wl)
    k, _ = q.autotune(wl.gates, wl.n, 4, reps=1)
    ref = q.Plan(wl.gates, wl.n)
    tuned = q.Plan(wl.gates, wl.n, k=k)
    s0, z0 = ref.forward(p, x)
    s1, z1 = tuned.forward(p, x)
    d0 = ref.backward(g)
    d1 = tuned.backward(g)
    torch.cuda.synchronize()
    t = TOL["c64"]
    assert np.abs((z1 - z0).cpu().numpy()).max() <= t["z"]
    assert np.abs((s1 - s0).cpu().numpy()).max() <= t["state"]
    check_grad(d1[0].cpu().numpy(), d0[0].cpu().numpy(), "c64", "dparams")
    check_grad(d1[1].cpu().numpy(), d0[1].cpu().numpy(), "c64", "dinputs")


def test_multi_autotune_per_qubit_count(q):
    wls = W.multi_circuit_config(n_circuits=6, n_min=9, n_max=15, d_min=1, d_max=2, seed=5)
    circuits = [(w.gates, w.n) for w in wls]
    ks = q.multi_autotune(circuits, 2, reps=1)
    assert len(ks) == len(wls)
    for w, k in zip(wls, ks):   # multi-circuit tiles hold at most 11 qubits (complex64)
        if w.n <= 11:
            assert k == w.n
        else:
            assert k in (9, 10, 11)
    by_n = {}
    for w, k in zip(wls, ks):
        assert by_n.setdefault(w.n, k) == k
    # the plan accepts them and runs
    B = 2
    mp = q.MultiPlan(circuits, ks=ks)
    rd = torch.float32
    p = torch.tensor(np.concatenate([w.params for w in wls]), dtype=rd, device="cuda")
    x = torch.tensor(np.concatenate([w.inputs[:B].ravel() for w in wls]), dtype=rd, device="cuda")
    ref = q.MultiPlan(circuits)
    _, z1 = mp.forward(p, x, B)
    _, z0 = ref.forward(p, x, B)
    torch.cuda.synchronize()
    assert mp.sync_status() == 0
    assert np.abs((z1 - z0).cpu().numpy()).max() <= TOL["c64"]["z"]
