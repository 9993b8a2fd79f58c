"""Writes the stored oracle values under tests/golden/ (calls only oracle/ and workloads/).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    wl = W.config(1)
    psi = oracle.simulate_kron(wl.gates, wl.n, wl.params, wl.inputs)
    z = oracle.expval_z(psi, wl.n)
    with open(os.path.join(HERE, "c1_z.txt"), "w") as f:
        f.write("# <Z_i> of workload C1 (4 qubits, batch 8), FP64 Kronecker oracle; rows = samples\n")
        for row in z:
            f.write(" ".join(f"{v:.17e}" for v in row) + "\n")
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out)
    with open(os.path.join(HERE, "c1_grad.txt"), "w") as f:
        f.write("# parameter-shift dL/dparams (16) then dL/dinputs (8x4) of C1 with its seeded grad_out\n")
        f.write(" ".join(f"{v:.17e}" for v in dp) + "\n")
        for row in di:
            f.write(" ".join(f"{v:.17e}" for v in row) + "\n")


if __name__ == "__main__":
    main()
