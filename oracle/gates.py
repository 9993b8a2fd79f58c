"""Gate matrices and their Kronecker expansion (Sec. "Gate Matrix Caching").

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

Conventions (Secs. "Symbols" and "Concept of Shapes" of the paper): qubit w is the w-th most significant bit of an
amplitude index, so on W qubits a single-qubit gate G on qubit w is I_{2^w} (x) G (x) I_{2^(W-1-w)}.
The printed exponent in Eq. 2 (I_{2^(W-w)} after the gate) would give dimension 2^(W+1); the reading
used here is the 0-based one that keeps the dimension at 2^W.
"""
from __future__ import annotations

import numpy as np

# gate codes, identical to the public enum
RX, RY, RZ, H, X, CNOT, CZ = range(7)

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)   # |0><0|
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)   # |1><1|


def rx(theta: float) -> np.ndarray:
    """R_x(theta) as the sum of two cached partial matrices (Eq. 1):
    R_xa cos(theta/2) + R_xb (-i sin(theta/2)), with R_xa = I and R_xb = X."""
    return I2 * np.cos(theta / 2) + PX * (-1j * np.sin(theta / 2))


def ry(theta: float) -> np.ndarray:
    """R_y(theta) = exp(-i theta Y / 2) = I cos(theta/2) - i Y sin(theta/2), the same two-partial
    decomposition as Eq. 1 with Y in place of X (the paper names only R_x)."""
    return I2 * np.cos(theta / 2) + PY * (-1j * np.sin(theta / 2))


def rz(theta: float) -> np.ndarray:
    """R_z(theta) = exp(-i theta Z / 2) = diag(e^{-i theta/2}, e^{+i theta/2})."""
    return I2 * np.cos(theta / 2) + PZ * (-1j * np.sin(theta / 2))


def hadamard() -> np.ndarray:
    return (PX + PZ) / np.sqrt(2.0)


def pauli_x() -> np.ndarray:
    return PX.copy()


def gate_angle(g, params, inputs_row):
    """Angle of a parametric gate: params[p] for p >= 0, inputs_row[-2 - p] for p <= -2."""
    p = g[3]
    if p >= 0:
        return float(params[p])
    if p <= -2:
        return float(inputs_row[-2 - p])
    raise ValueError("gate has no parameter")


def gate_matrix_2x2(kind: int, angle: float | None = None) -> np.ndarray:
    if kind == RX:
        return rx(angle)
    if kind == RY:
        return ry(angle)
    if kind == RZ:
        return rz(angle)
    if kind == H:
        return hadamard()
    if kind == X:
        return pauli_x()
    raise ValueError(f"not a single-qubit gate: {kind}")


def expand_1q(G: np.ndarray, w: int, W: int) -> np.ndarray:
    """Eq. 2: I_{2^w} (x) G (x) I_{2^(W-1-w)}, qubits before the gate on the left."""
    return np.kron(np.kron(np.eye(2 ** w, dtype=np.complex128), G),
                   np.eye(2 ** (W - 1 - w), dtype=np.complex128))


def _kron_chain(factors):
    out = np.ones((1, 1), dtype=np.complex128)
    for f in factors:
        out = np.kron(out, f)
    return out


def expand_controlled(c: int, t: int, U: np.ndarray, W: int) -> np.ndarray:
    """Controlled-U with control qubit c and target t on W qubits, written as
    P0_c (x) I + P1_c (x) U_t with identities on every other qubit, factors in qubit order."""
    if c == t:
        raise ValueError("control equals target")
    f0 = [P0 if q == c else I2 for q in range(W)]
    f1 = [P1 if q == c else (U if q == t else I2) for q in range(W)]
    return _kron_chain(f0) + _kron_chain(f1)


def full_gate_matrix(g, W: int, params, inputs_row) -> np.ndarray:
    """Dense 2^W x 2^W matrix of one gate tuple (type, targets, controls, param)."""
    kind, targets, controls, _ = g
    if kind in (RX, RY, RZ):
        return expand_1q(gate_matrix_2x2(kind, gate_angle(g, params, inputs_row)), targets[0], W)
    if kind in (H, X):
        return expand_1q(gate_matrix_2x2(kind), targets[0], W)
    if kind == CNOT:
        return expand_controlled(controls[0], targets[0], PX, W)
    if kind == CZ:
        return expand_controlled(controls[0], targets[0], PZ, W)
    raise ValueError(f"unknown gate type {kind}")
