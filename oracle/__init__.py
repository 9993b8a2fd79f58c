"""FP64 CPU oracle for batched parameterised-circuit simulation — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs may
import this package. The library's product path never calls it and shares no code with it.

It computes, plainly and slowly, what the accelerated path computes:

* ``gates``     2x2 gate matrices (RX via the paper's partial-matrix decomposition, Eq. 1) and their
                Kronecker expansion to the full register (Eq. 2, reading: I_{2^w} (x) G (x) I_{2^(W-1-w)}
                with 0-based w, MSb-0 as in Sec. "Symbols").
* ``kron``      Oracle-K: every gate expanded to a dense 2^W x 2^W matrix by explicit Kronecker
                products and applied by a dense matrix-vector product (Sec. "Gate Matrix Caching", Eq. 2).
* ``strided``   Oracle-S: every gate applied by reshaping the state to (2^w, 2, 2^(W-1-w)) and
                contracting the middle axis (the reshape method of Sec. "Concept of Shapes"); used above 12 qubits.
* ``measure``   <Z_i> = sum_x |psi_x|^2 (1 - 2 bit_i(x)) (measurement layer, Sec. "Hybrid Machine Learning").
* ``grad``      loss L = sum_{b,i} g_{b,i} <Z_i>_b, its gradient by the parameter-shift rule
                (exact for exp(-i theta P / 2)) and by central finite differences (Sec. "Hybrid Machine Learning"
                mentions both; the reading that the shift rule is exact, not a finite difference,
                is recorded in the design notes).
* ``adjoint``   the same gradient by the adjoint sweep (psi and lambda uncomputed gate by gate, FP64);
                pinned against the exact parameter shift, it gives every gradient entry at 20+ qubits.
* ``bitsim``    a pure-Python per-basis-index simulator used only to pin the other two on tiny inputs.
* ``remapping`` quantum weight remapping angle = pi * tanh(weight) and its chain rule (Sec. "Additional Optimizations").

Every function here is pinned by tests in ``tests/test_oracle_pins.py`` against closed forms,
library routines (scipy ``expm``) and brute force; none is "parity unpinned".
"""
from .gates import (gate_matrix_2x2, expand_1q, expand_controlled, full_gate_matrix,
                    rx, ry, rz, hadamard, pauli_x, gate_angle)
from .kron import simulate_kron
from .strided import simulate_strided
from .measure import expval_z, expval_zz
from .grad import loss, grad_param_shift, grad_finite_diff, forward_z
from .adjoint import grad_adjoint
from .remapping import remap, remap_slope, forward_z_remapped, grad_remapped

__all__ = ["gate_matrix_2x2", "expand_1q", "expand_controlled", "full_gate_matrix", "rx", "ry",
           "rz", "hadamard", "pauli_x", "gate_angle", "simulate_kron", "simulate_strided",
           "expval_z", "expval_zz", "loss", "grad_param_shift", "grad_finite_diff", "forward_z", "grad_adjoint",
           "remap", "remap_slope", "forward_z_remapped", "grad_remapped"]
