"""Seeded synthetic workloads: circuit descriptions and the random draws that feed them.

This module holds no simulation arithmetic. It only builds gate lists (as plain tuples) and
draws inputs, parameters and loss weights from a counter-based generator, so that the FP64
oracle and the CUDA path can be fed byte-identical problems without sharing any code.

Gate tuples mirror the C struct ``qsim_gate``: ``(type, targets, controls, param)`` where
``targets``/``controls`` are 2-tuples with -1 for unused slots and ``param`` is

* ``>= 0``  index into the trainable parameter vector,
* ``-1``    no parameter (H, X, CNOT, CZ),
* ``<= -2`` input column ``-2 - param`` of the per-sample input matrix.

Qubit ``q`` is the ``q``-th most significant bit of an amplitude index (MSb-0 ordering of the
paper's Sec. "Symbols"); that convention is the simulators' business, not this module's.

The five standard workloads follow the paper's hybrid-model structure (Sec. "Hybrid Machine Learning": an
embedding layer, trainable rotation layers, a measurement layer):

=====  ==========================================================================
C1     4 qubits, batch 8, complex128, RX encoding + 2 x (RY, RZ per qubit + CNOT ring)
C2     12 qubits, batch 1024, complex64, RX encoding + 6 layers
C3     20 qubits, batch 64, complex64, RX encoding + 10 layers (forward + backward)
C4     256 circuits, 8..22 qubits (log-uniform), depth 4..16, RY/RZ + CZ ladder, batch 4
C5     30 qubits, batch 1, complex64, RX encoding + 8 layers (forward + backward)
=====  ==========================================================================
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# gate type codes (same values as the C enum)
RX, RY, RZ, H, X, CNOT, CZ = range(7)
GATE_NAMES = {RX: "rx", RY: "ry", RZ: "rz", H: "h", X: "x", CNOT: "cx", CZ: "cz"}
PARAMETRIC = (RX, RY, RZ)

_MASK64 = (1 << 64) - 1
SEED_BASE = 0x240409213


class SplitMix64:
    """Counter-based splitmix64 stream (Steele, Lea, Flood 2014), exact 64-bit arithmetic.

    ``uniform()`` maps the top 53 bits to [0, 1): u = (x >> 11) * 2**-53.
    """

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, count: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(count)], dtype=np.float64)


def gate(kind: int, targets=(-1, -1), controls=(-1, -1), param: int = -1):
    t = tuple(targets) + (-1,) * (2 - len(targets))
    c = tuple(controls) + (-1,) * (2 - len(controls))
    return (int(kind), (int(t[0]), int(t[1])), (int(c[0]), int(c[1])), int(param))


def input_param(col: int) -> int:
    """Encode input column ``col`` in the ``param`` field."""
    return -2 - col


def ring_ansatz(n: int, layers: int, encode: bool = True):
    """RX angle encoding of n inputs, then ``layers`` x (RY(q), RZ(q) for all q, CNOT ring).

    Layer l uses parameter l*2n+q for RY(q) and l*2n+n+q for RZ(q); the ring is
    CNOT(q, (q+1) mod n) for q = 0..n-1 in that order.
    """
    gates = []
    if encode:
        gates += [gate(RX, (q,), param=input_param(q)) for q in range(n)]
    for l in range(layers):
        gates += [gate(RY, (q,), param=l * 2 * n + q) for q in range(n)]
        gates += [gate(RZ, (q,), param=l * 2 * n + n + q) for q in range(n)]
        if n >= 2:
            gates += [gate(CNOT, ((q + 1) % n,), (q,)) for q in range(n)]
    return gates


def hea_cz_ansatz(n: int, depth: int, encode: bool = True):
    """Hardware-efficient ansatz: RX encoding, then depth x (RY(q), RZ(q) all q, CZ(q,q+1) ladder)."""
    gates = []
    if encode:
        gates += [gate(RX, (q,), param=input_param(q)) for q in range(n)]
    for l in range(depth):
        gates += [gate(RY, (q,), param=l * 2 * n + q) for q in range(n)]
        gates += [gate(RZ, (q,), param=l * 2 * n + n + q) for q in range(n)]
        gates += [gate(CZ, (q + 1,), (q,)) for q in range(n - 1)]
    return gates


def sel_ansatz(n: int, layers: int, reupload: bool = False, encode: bool = True):
    """Strongly Entangling Layers (the circuit family of the paper's App. "Barren Plateaus").

    Layer l: Rot(phi, theta, omega) = RZ(omega) RY(theta) RZ(phi) on every qubit q (applied as RZ(phi),
    then RY(theta), then RZ(omega); parameters 3(l n + q) + 0, 1, 2), then CNOT(q, (q + r) mod n) for
    q = 0..n-1 with range r = (l mod (n - 1)) + 1. ``encode``: RX(x_q) angle encoding of n inputs
    before the first layer; ``reupload``: before every layer (data re-uploading, the embedding
    variant named in the paper's Sec. "Hybrid Machine Learning").
    """
    gates = []
    for l in range(layers):
        if encode and (l == 0 or reupload):
            gates += [gate(RX, (q,), param=input_param(q)) for q in range(n)]
        for q in range(n):
            base = 3 * (l * n + q)
            gates += [gate(RZ, (q,), param=base), gate(RY, (q,), param=base + 1), gate(RZ, (q,), param=base + 2)]
        if n >= 2:
            r = (l % (n - 1)) + 1
            gates += [gate(CNOT, ((q + r) % n,), (q,)) for q in range(n)]
    return gates


def sel_workload(name: str, n: int, batch: int, layers: int, dtype: str, seed: int, reupload: bool = True,
                 encode: bool = True) -> Workload:
    gates = sel_ansatz(n, layers, reupload, encode)
    rng = SplitMix64(seed)
    inputs, params, grad_out = _draw(rng, batch, n if encode else 0, count_params(gates), n)
    return Workload(name, n, batch, dtype, gates, params, inputs, grad_out, True,
                    {"layers": layers, "seed": seed, "reupload": reupload})


def count_params(gates) -> int:
    return 1 + max([g[3] for g in gates if g[3] >= 0], default=-1)


def count_inputs(gates) -> int:
    return 1 + max([-2 - g[3] for g in gates if g[3] <= -2], default=-1)


@dataclass
class Workload:
    name: str
    n: int
    batch: int
    dtype: str                      # "c64" or "c128"
    gates: list
    params: np.ndarray              # (P,) float64
    inputs: np.ndarray              # (B, n_in) float64
    grad_out: np.ndarray            # (B, n) float64
    backward: bool = True
    meta: dict = field(default_factory=dict)

    @property
    def n_params(self):
        return len(self.params)

    @property
    def n_inputs(self):
        return self.inputs.shape[1]


def _draw(rng: SplitMix64, batch: int, n_in: int, n_par: int, n_out: int):
    inputs = rng.uniforms(batch * n_in).reshape(batch, n_in) * math.pi
    params = rng.uniforms(n_par) * (2.0 * math.pi)
    grad_out = rng.uniforms(batch * n_out).reshape(batch, n_out) * 2.0 - 1.0
    return inputs, params, grad_out


def ring_workload(name: str, n: int, batch: int, layers: int, dtype: str, seed: int,
                  backward: bool = True) -> Workload:
    gates = ring_ansatz(n, layers)
    rng = SplitMix64(seed)
    inputs, params, grad_out = _draw(rng, batch, n, count_params(gates), n)
    return Workload(name, n, batch, dtype, gates, params, inputs, grad_out, backward,
                    {"layers": layers, "seed": seed})


def config(c: int, **overrides) -> Workload:
    """Standard workloads C1, C2, C3, C5 (C4 is a list: see :func:`multi_circuit_config`).

    ``overrides`` may change ``n``, ``batch``, ``layers`` or ``dtype`` to get a smaller instance of
    the same ansatz with the same seed (for example the 12-qubit version of C3/C5).
    """
    table = {
        1: dict(n=4, batch=8, layers=2, dtype="c128", backward=False),
        2: dict(n=12, batch=1024, layers=6, dtype="c64", backward=False),
        3: dict(n=20, batch=64, layers=10, dtype="c64", backward=True),
        5: dict(n=30, batch=1, layers=8, dtype="c64", backward=True),
    }
    if c not in table:
        raise ValueError(f"no single-circuit config C{c}")
    spec = dict(table[c])
    spec.update(overrides)
    return ring_workload(f"C{c}", spec["n"], spec["batch"], spec["layers"], spec["dtype"],
                         SEED_BASE + c, spec["backward"])


def multi_circuit_config(n_circuits: int = 256, batch: int = 4, n_min: int = 8, n_max: int = 22,
                         d_min: int = 4, d_max: int = 16, seed: int = SEED_BASE + 4):
    """C4: ``n_circuits`` hardware-efficient circuits of uneven size, one generator stream.

    Per circuit, in this order: n = floor(exp(ln n_min + u (ln(n_max+1) - ln n_min))),
    depth = d_min + floor((d_max - d_min + 1) u), then inputs (B x n) ~ U[0, pi),
    params (2 n depth) ~ U[0, 2 pi), grad_out (B x n) ~ U[-1, 1).
    """
    rng = SplitMix64(seed)
    out = []
    lo, hi = math.log(n_min), math.log(n_max + 1)
    for i in range(n_circuits):
        n = int(math.floor(math.exp(lo + rng.uniform() * (hi - lo))))
        n = min(max(n, n_min), n_max)
        depth = d_min + int(math.floor((d_max - d_min + 1) * rng.uniform()))
        depth = min(depth, d_max)
        gates = hea_cz_ansatz(n, depth)
        inputs, params, grad_out = _draw(rng, batch, n, count_params(gates), n)
        out.append(Workload(f"C4[{i}]", n, batch, "c64", gates, params, inputs, grad_out, True,
                            {"depth": depth}))
    return out


def gates_to_array(gates) -> np.ndarray:
    """(G, 6) int32 array in ``qsim_gate`` field order: type, t0, t1, c0, c1, param."""
    arr = np.zeros((len(gates), 6), dtype=np.int32)
    for i, (k, t, c, p) in enumerate(gates):
        arr[i] = (k, t[0], t[1], c[0], c[1], p)
    return arr
