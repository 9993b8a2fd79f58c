"""Oracle-S: per-gate strided simulation by reshaping (Sec. "Concept of Shapes").

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

The paper applies a single-qubit gate G on qubit w by viewing the state as (..., 2, ...) with the
w-th axis separate and multiplying by G over that axis. Here the batched state (B, 2^W) is viewed as
(B, 2^w, 2, 2^(W-1-w)) and the middle axis is contracted with G. Controlled gates act on the
sub-array where the control axis is 1. FP64 throughout; no blocking or fusion.
"""
from __future__ import annotations

import numpy as np

from .gates import gate_matrix_2x2, gate_angle, PX, PZ, RX, RY, RZ, H, X, CNOT, CZ
from .kron import initial_states


def _apply_1q(psi: np.ndarray, n: int, w: int, G: np.ndarray) -> np.ndarray:
    """psi (B, 2^n); G (2,2) shared or (B,2,2) per sample."""
    B = psi.shape[0]
    v = psi.reshape(B, 2 ** w, 2, 2 ** (n - 1 - w))
    a0 = v[:, :, 0, :].copy()
    a1 = v[:, :, 1, :].copy()
    if G.ndim == 2:
        v[:, :, 0, :] = G[0, 0] * a0 + G[0, 1] * a1
        v[:, :, 1, :] = G[1, 0] * a0 + G[1, 1] * a1
    else:
        g = G[:, :, :, None, None]
        v[:, :, 0, :] = g[:, 0, 0] * a0 + g[:, 0, 1] * a1
        v[:, :, 1, :] = g[:, 1, 0] * a0 + g[:, 1, 1] * a1
    return psi


def _apply_controlled(psi: np.ndarray, n: int, c: int, t: int, U: np.ndarray) -> np.ndarray:
    B = psi.shape[0]
    v = psi.reshape((B,) + (2,) * n)
    idx = [slice(None)] * (n + 1)
    idx[1 + c] = 1
    sub = v[tuple(idx)]                       # control axis fixed to 1; target axis shifts if t > c
    tt = t if t < c else t - 1
    sub_flat = np.moveaxis(sub, 1 + tt, -1)    # target axis last
    a0 = sub_flat[..., 0].copy()
    a1 = sub_flat[..., 1].copy()
    sub_flat[..., 0] = U[0, 0] * a0 + U[0, 1] * a1
    sub_flat[..., 1] = U[1, 0] * a0 + U[1, 1] * a1
    return psi


def simulate_strided(gates, n: int, params, inputs, init=None) -> np.ndarray:
    """Final states (B, 2^n) complex128; same contract as :func:`oracle.simulate_kron`."""
    inputs = np.atleast_2d(np.asarray(inputs, dtype=np.float64))
    batch = inputs.shape[0]
    psi = initial_states(n, batch, init)
    for g in gates:
        kind, targets, controls, p = g
        if kind in (RX, RY, RZ):
            if p <= -2:
                G = np.stack([gate_matrix_2x2(kind, gate_angle(g, params, inputs[b]))
                              for b in range(batch)])
            else:
                G = gate_matrix_2x2(kind, gate_angle(g, params, None))
            _apply_1q(psi, n, targets[0], G)
        elif kind in (H, X):
            _apply_1q(psi, n, targets[0], gate_matrix_2x2(kind))
        elif kind == CNOT:
            _apply_controlled(psi, n, controls[0], targets[0], PX)
        elif kind == CZ:
            _apply_controlled(psi, n, controls[0], targets[0], PZ)
        else:
            raise ValueError(f"unknown gate type {kind}")
    return psi
