"""Oracle-K: dense Kronecker-expanded simulation (Sec. "Gate Matrix Caching", Eq. 2).

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

Each gate is expanded to its full 2^W x 2^W matrix and applied to every state by a dense product,
in circuit order. Gates whose angle is shared by the whole batch are applied to all samples at once
((2^W x 2^W) @ (2^W x B)); gates driven by an input column get one matrix per sample. Practical up
to about 12 qubits (a 12-qubit gate matrix is 256 MiB).
"""
from __future__ import annotations

import numpy as np

from .gates import full_gate_matrix


def initial_states(n: int, batch: int, init=None) -> np.ndarray:
    """|0...0> for every sample, or a copy of ``init`` (B, 2^n)."""
    if init is not None:
        psi = np.array(init, dtype=np.complex128).reshape(batch, 2 ** n).copy()
        return psi
    psi = np.zeros((batch, 2 ** n), dtype=np.complex128)
    psi[:, 0] = 1.0
    return psi


def simulate_kron(gates, n: int, params, inputs, init=None, max_qubits: int = 13) -> np.ndarray:
    """Final states (B, 2^n) complex128 of the gate list applied to the batch."""
    if n > max_qubits:
        raise ValueError(f"dense Kronecker oracle limited to {max_qubits} qubits")
    inputs = np.atleast_2d(np.asarray(inputs, dtype=np.float64))
    batch = inputs.shape[0]
    psi = initial_states(n, batch, init)
    for g in gates:
        if g[3] <= -2:
            for b in range(batch):
                U = full_gate_matrix(g, n, params, inputs[b])
                psi[b] = U @ psi[b]
        else:
            U = full_gate_matrix(g, n, params, inputs[0] if batch else None)
            psi = (U @ psi.T).T
    return psi
