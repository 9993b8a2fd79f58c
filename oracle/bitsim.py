"""Brute-force per-basis-index simulator (pure Python loops) for pinning the oracle on tiny inputs.

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

It applies each gate by walking every amplitude index and reading the target/control bits with
integer shifts (bit of qubit q = (x >> (n-1-q)) & 1, MSb-0 as in Sec. "Symbols"). It shares no
array reshaping or Kronecker code with ``kron`` / ``strided``; only the 2x2 matrices are reused.
"""
from __future__ import annotations

from .gates import gate_matrix_2x2, gate_angle, RX, RY, RZ, H, X, CNOT, CZ


def simulate_bits(gates, n, params, inputs_row, init=None):
    dim = 1 << n
    psi = [0j] * dim
    if init is None:
        psi[0] = 1 + 0j
    else:
        psi = [complex(v) for v in init]
    for g in gates:
        kind, targets, controls, p = g
        new = list(psi)
        if kind in (RX, RY, RZ, H, X):
            ang = gate_angle(g, params, inputs_row) if kind in (RX, RY, RZ) else None
            G = gate_matrix_2x2(kind, ang)
            sh = n - 1 - targets[0]
            for x in range(dim):
                b = (x >> sh) & 1
                x0 = x & ~(1 << sh)
                x1 = x | (1 << sh)
                new[x] = complex(G[b, 0]) * psi[x0] + complex(G[b, 1]) * psi[x1]
        elif kind == CNOT:
            sc, st = n - 1 - controls[0], n - 1 - targets[0]
            for x in range(dim):
                new[x] = psi[x ^ (1 << st)] if (x >> sc) & 1 else psi[x]
        elif kind == CZ:
            sa, sb = n - 1 - controls[0], n - 1 - targets[0]
            for x in range(dim):
                new[x] = -psi[x] if ((x >> sa) & 1) and ((x >> sb) & 1) else psi[x]
        else:
            raise ValueError(kind)
        psi = new
    return psi


def expval_z_bits(psi, n):
    out = []
    for i in range(n):
        sh = n - 1 - i
        out.append(sum(abs(a) ** 2 * (1 - 2 * ((x >> sh) & 1)) for x, a in enumerate(psi)))
    return out
