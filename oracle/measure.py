"""Measurement layer (Sec. "Hybrid Machine Learning"): Pauli-Z expectation values of every qubit.

Test infrastructure only (the FP64 oracle): the library's product path never imports it.

<Z_i>_b = sum_x |psi_b[x]|^2 (1 - 2 bit_i(x)), where bit_i(x) is the i-th most significant of the n
index bits (MSb-0, Sec. "Symbols"), i.e. (x >> (n-1-i)) & 1.
"""
from __future__ import annotations

import numpy as np


def expval_z(psi: np.ndarray, n: int) -> np.ndarray:
    psi = np.atleast_2d(psi)
    prob = np.abs(psi) ** 2                        # (B, 2^n)
    x = np.arange(2 ** n)
    out = np.empty((psi.shape[0], n), dtype=np.float64)
    for i in range(n):
        sign = 1.0 - 2.0 * ((x >> (n - 1 - i)) & 1)
        out[:, i] = prob @ sign
    return out


def expval_zz(psi: np.ndarray, n: int, i: int, j: int) -> np.ndarray:
    """<Z_i Z_j> per sample (used only by the oracle's own GHZ self-check)."""
    psi = np.atleast_2d(psi)
    prob = np.abs(psi) ** 2
    x = np.arange(2 ** n)
    si = 1.0 - 2.0 * ((x >> (n - 1 - i)) & 1)
    sj = 1.0 - 2.0 * ((x >> (n - 1 - j)) & 1)
    return prob @ (si * sj)
