"""Helpers shared by the GPU tests: workload -> CUDA tensors, tolerance checks, oracle gradients."""
import numpy as np
import torch

import oracle
import workloads as W

TOL = {"c64": dict(z=1e-5, state=1e-5, grad_rel=1e-4, grad_abs=1e-7),
       "c128": dict(z=1e-12, state=1e-12, grad_rel=1e-12, grad_abs=1e-14)}


def tensors(wl, dtype=None, device="cuda"):
    dt = torch.float64 if (dtype or wl.dtype) == "c128" else torch.float32
    p = torch.tensor(wl.params, dtype=dt, device=device)
    x = torch.tensor(wl.inputs, dtype=dt, device=device)
    g = torch.tensor(wl.grad_out, dtype=torch.float64, device=device)
    return p, x, g


def rounded(wl, dtype):
    """Angles as the GPU sees them (float32 in c64 mode): the oracle must use the same values."""
    if dtype == "c64":
        return wl.params.astype(np.float32).astype(np.float64), wl.inputs.astype(np.float32).astype(np.float64)
    return wl.params, wl.inputs


def check_grad(got, ref, dtype, what=""):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    t = TOL[dtype]
    if ref.size == 0:
        return
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    nrm = np.linalg.norm(ref)
    rel = np.linalg.norm(got - ref) / nrm if nrm > 0 else np.linalg.norm(got - ref)
    assert rel <= t["grad_rel"], f"{what}: norm-wise relative gradient error {rel:.3e}"
    assert err.max() <= t["grad_rel"] * scale + t["grad_abs"], f"{what}: max abs error {err.max():.3e} (scale {scale:.3e})"


def random_circuit(rng, n, g, n_params=6, n_inputs=2):
    out = []
    for _ in range(g):
        k = int(rng.integers(0, 7))
        if k in (W.RX, W.RY, W.RZ):
            if n_inputs > 0 and rng.uniform() < 0.3:
                p = W.input_param(int(rng.integers(0, n_inputs)))
            else:
                p = int(rng.integers(0, n_params))
            out.append(W.gate(k, (int(rng.integers(0, n)),), param=p))
        elif k in (W.H, W.X):
            out.append(W.gate(k, (int(rng.integers(0, n)),)))
        elif n >= 2:
            c, t = rng.choice(n, 2, replace=False)
            out.append(W.gate(k, (int(t),), (int(c),)))
    return out


def shift_grad_strided(gates, n, params, inputs, grad_out, which, prefix=None):
    """Parameter-shift derivative of sum(g * z) w.r.t. the angle of gate ``which`` only, evaluated on
    the split circuit prefix | gate | suffix. ``prefix`` = (index, state after gates[:index]) lets
    several calls share the prefix. Returns the per-sample derivative (B,)."""
    if prefix is not None and prefix[0] <= which:
        pre = oracle.simulate_strided(gates[prefix[0]:which], n, params, inputs, init=prefix[1])
    else:
        pre = oracle.simulate_strided(gates[:which], n, params, inputs)
    g = gates[which]
    vals = []
    for delta in (np.pi / 2, -np.pi / 2):
        params2 = np.concatenate([params, [0.0]])
        inputs2 = np.array(inputs, copy=True)
        if g[3] >= 0:
            params2[-1] = params[g[3]] + delta
            gs = (g[0], g[1], g[2], len(params2) - 1)
        else:
            col = -2 - g[3]
            inputs2 = np.concatenate([inputs2, inputs2[:, col:col + 1] + delta], axis=1)
            gs = (g[0], g[1], g[2], -2 - (inputs2.shape[1] - 1))
        psi = oracle.simulate_strided([gs] + list(gates[which + 1:]), n, params2, inputs2, init=pre)
        vals.append(np.sum(grad_out * oracle.expval_z(psi, n), axis=1))
    return (vals[0] - vals[1]) / 2
