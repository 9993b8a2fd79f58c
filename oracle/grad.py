"""Loss and reference gradients (Sec. "Hybrid Machine Learning": parameter-shift rule and backpropagation).

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

L = sum_{b,i} g_{b,i} <Z_i>_b. Trainable parameters are shared by the batch, so dL/dparams sums
over samples; encoded inputs belong to one sample each, so dL/dinputs is per sample.

* Parameter shift: every rotation is exp(-i theta P / 2) with P a Pauli, for which
  d<O>/d theta = (<O>(theta + pi/2) - <O>(theta - pi/2)) / 2 exactly. A parameter used by several
  gates gets the sum over its occurrences, each shifted on its own.
* Central finite differences with step h (FP64): (L(p + h) - L(p - h)) / (2 h), moving every
  occurrence of the parameter together.
"""
from __future__ import annotations

import math

import numpy as np

from .kron import simulate_kron
from .strided import simulate_strided
from .measure import expval_z


def _sim(method):
    return {"kron": simulate_kron, "strided": simulate_strided}[method]


def forward_z(gates, n, params, inputs, method="kron", init=None):
    return expval_z(_sim(method)(gates, n, params, inputs, init=init), n)


def loss(z: np.ndarray, grad_out: np.ndarray) -> float:
    return float(np.sum(np.asarray(grad_out) * z))


def _per_sample_loss(gates, n, params, inputs, grad_out, method, init=None):
    z = forward_z(gates, n, params, inputs, method, init)
    return np.sum(np.asarray(grad_out) * z, axis=1)          # (B,)


def _shifted_eval(gates, n, params, inputs, grad_out, k, delta, method, init):
    """Per-sample loss with gate k's angle moved by delta (only that occurrence)."""
    g = gates[k]
    params2 = np.concatenate([np.asarray(params, dtype=np.float64), [0.0]])
    extra = len(params2) - 1
    p = g[3]
    if p >= 0:
        params2[extra] = params2[p] + delta
        gates2 = list(gates)
        gates2[k] = (g[0], g[1], g[2], extra)
        return _per_sample_loss(gates2, n, params2, inputs, grad_out, method, init)
    # input-driven gate: shift that sample column for every sample at once (samples are independent)
    col = -2 - p
    inputs2 = np.array(inputs, dtype=np.float64, copy=True)
    inputs2 = np.concatenate([inputs2, inputs2[:, col:col + 1] + delta], axis=1)
    gates2 = list(gates)
    gates2[k] = (g[0], g[1], g[2], -2 - (inputs2.shape[1] - 1))
    return _per_sample_loss(gates2, n, params, inputs2, grad_out, method, init)


def grad_param_shift(gates, n, params, inputs, grad_out, method="kron", init=None,
                     param_subset=None, input_subset=None):
    """(dparams (P,), dinputs (B, n_in)) by the exact +-pi/2 shift rule, summed over occurrences.

    ``param_subset`` / ``input_subset`` restrict which entries are evaluated (others are NaN).
    """
    inputs = np.atleast_2d(np.asarray(inputs, dtype=np.float64))
    P = len(params)
    n_in = inputs.shape[1]
    dparams = np.zeros(P)
    dinputs = np.zeros(inputs.shape)
    want_p = set(range(P)) if param_subset is None else set(param_subset)
    want_i = set(range(n_in)) if input_subset is None else set(input_subset)
    for k, g in enumerate(gates):
        p = g[3]
        if p == -1:
            continue
        if p >= 0 and p not in want_p:
            continue
        if p <= -2 and (-2 - p) not in want_i:
            continue
        lp = _shifted_eval(gates, n, params, inputs, grad_out, k, math.pi / 2, method, init)
        lm = _shifted_eval(gates, n, params, inputs, grad_out, k, -math.pi / 2, method, init)
        d = (lp - lm) / 2.0
        if p >= 0:
            dparams[p] += d.sum()
        else:
            dinputs[:, -2 - p] += d
    for p in range(P):
        if p not in want_p:
            dparams[p] = np.nan
    for c in range(n_in):
        if c not in want_i:
            dinputs[:, c] = np.nan
    return dparams, dinputs


def grad_finite_diff(gates, n, params, inputs, grad_out, h=1e-4, method="kron", init=None,
                     param_subset=None, input_subset=None):
    """Central differences in FP64: every occurrence of a parameter moves together."""
    inputs = np.atleast_2d(np.asarray(inputs, dtype=np.float64))
    params = np.asarray(params, dtype=np.float64)
    P = len(params)
    n_in = inputs.shape[1]
    dparams = np.full(P, np.nan)
    dinputs = np.full(inputs.shape, np.nan)
    for p in (range(P) if param_subset is None else param_subset):
        pp = params.copy(); pp[p] += h
        pm = params.copy(); pm[p] -= h
        lp = _per_sample_loss(gates, n, pp, inputs, grad_out, method, init).sum()
        lm = _per_sample_loss(gates, n, pm, inputs, grad_out, method, init).sum()
        dparams[p] = (lp - lm) / (2 * h)
    for c in (range(n_in) if input_subset is None else input_subset):
        ip = inputs.copy(); ip[:, c] += h
        im = inputs.copy(); im[:, c] -= h
        lp = _per_sample_loss(gates, n, params, ip, grad_out, method, init)
        lm = _per_sample_loss(gates, n, params, im, grad_out, method, init)
        dinputs[:, c] = (lp - lm) / (2 * h)
    return dparams, dinputs
