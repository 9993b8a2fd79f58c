"""Adjoint-method gradient of L = sum_{b,i} g_{b,i} <Z_i>_b in FP64 (the reverse-mode derivative the
paper obtains by backpropagation, Sec. "Hybrid Machine Learning", written as the adjoint sweep over
the gate list).

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

Definitions. psi_k is the state after gate k (psi_L the final state), O_b = sum_i g_{b,i} Z_i, and
lambda_k = U_{k+1}^dag ... U_L^dag O_b psi_L. For a rotation U_k = exp(-i theta P / 2),
d psi_L / d theta = U_L ... U_{k+1} (-i/2) P psi_k, so

    dL/d theta_k = 2 Re <lambda_k | (-i/2) P | psi_k> = Im <lambda_k | P | psi_k>.

The sweep starts from psi_L and lambda_L = O psi_L and walks the gates backwards: the gradient of
gate k, then psi and lambda are both multiplied by U_k^dag. Every step uses the strided per-gate
application of Oracle-S (the reshape method of Sec. "Concept of Shapes"); no fusion or reordering.
Shared parameters sum over samples and occurrences; inputs are per sample.
"""
from __future__ import annotations

import numpy as np

from .gates import gate_matrix_2x2, gate_angle, PX, PY, PZ, RX, RY, RZ, H, X, CNOT, CZ
from .strided import simulate_strided, _apply_1q, _apply_controlled

_PAULI = {RX: PX, RY: PY, RZ: PZ}


def _loss_observable(psi: np.ndarray, n: int, grad_out: np.ndarray) -> np.ndarray:
    """lambda = (sum_i g_{b,i} Z_i) psi, Z_i diagonal with entries 1 - 2 bit_i(x) (MSb-0)."""
    x = np.arange(2 ** n)
    d = np.zeros((psi.shape[0], 2 ** n))
    for i in range(n):
        d += np.outer(grad_out[:, i], 1.0 - 2.0 * ((x >> (n - 1 - i)) & 1))
    return d * psi


def _gate_dagger(g, params, inputs, batch):
    """2x2 matrix of U^dag for a single-qubit gate: shared (2,2) or per sample (B,2,2)."""
    kind = g[0]
    if kind in (RX, RY, RZ):
        if g[3] <= -2:
            return np.stack([gate_matrix_2x2(kind, gate_angle(g, params, inputs[b])).conj().T
                             for b in range(batch)])
        return gate_matrix_2x2(kind, gate_angle(g, params, None)).conj().T
    return gate_matrix_2x2(kind).conj().T


def grad_adjoint(gates, n: int, params, inputs, grad_out, init=None):
    """(dparams (P,), dinputs (B, n_in)) by the adjoint sweep; same contract as grad_param_shift."""
    inputs = np.atleast_2d(np.asarray(inputs, dtype=np.float64))
    grad_out = np.atleast_2d(np.asarray(grad_out, dtype=np.float64))
    batch = inputs.shape[0]
    psi = simulate_strided(gates, n, params, inputs, init=init)
    lam = _loss_observable(psi, n, grad_out)
    dparams = np.zeros(len(params))
    dinputs = np.zeros(inputs.shape)
    for g in reversed(gates):
        kind, targets, controls, p = g
        if kind in (RX, RY, RZ):
            ppsi = _apply_1q(psi.copy(), n, targets[0], _PAULI[kind])
            gk = np.imag(np.sum(np.conj(lam) * ppsi, axis=1))          # Im <lambda|P|psi>, per sample
            if p >= 0:
                dparams[p] += gk.sum()
            else:
                dinputs[:, -2 - p] += gk
        if kind in (RX, RY, RZ, H, X):
            Ud = _gate_dagger(g, params, inputs, batch)
            _apply_1q(psi, n, targets[0], Ud)
            _apply_1q(lam, n, targets[0], Ud)
        elif kind in (CNOT, CZ):                                        # both are their own inverse
            U = PX if kind == CNOT else PZ
            _apply_controlled(psi, n, controls[0], targets[0], U)
            _apply_controlled(lam, n, controls[0], targets[0], U)
        else:
            raise ValueError(f"unknown gate type {kind}")
    return dparams, dinputs
