"""Quantum weight remapping (Sec. "Additional Optimizations") — test infrastructure only.

The paper maps every trainable weight into a bounded range such as [-pi, pi] with a smooth function,
naming the hyperbolic tangent; the reading taken here is angle = pi * tanh(weight), applied to the
trainable parameters only (encoded inputs are data, not weights). Gradients with respect to the raw
weights follow by the chain rule: dL/dw = dL/dangle * pi * (1 - tanh(w)^2).
"""
from __future__ import annotations

import numpy as np

from .grad import forward_z, grad_param_shift


def remap(weights):
    """pi * tanh(w), elementwise (FP64)."""
    return np.pi * np.tanh(np.asarray(weights, dtype=np.float64))


def remap_slope(weights):
    """d remap / d w = pi * (1 - tanh(w)^2)."""
    t = np.tanh(np.asarray(weights, dtype=np.float64))
    return np.pi * (1.0 - t * t)


def forward_z_remapped(gates, n, weights, inputs, method="kron", init=None):
    """<Z_i> of the circuit whose trainable angles are remap(weights)."""
    return forward_z(gates, n, remap(weights), inputs, method, init)


def grad_remapped(gates, n, weights, inputs, grad_out, method="kron", init=None, param_subset=None,
                  input_subset=None):
    """(dL/dweights, dL/dinputs): the exact shift rule at the remapped angles, then the chain rule."""
    dang, dinp = grad_param_shift(gates, n, remap(weights), inputs, grad_out, method, init,
                                  param_subset, input_subset)
    return dang * remap_slope(weights), dinp
