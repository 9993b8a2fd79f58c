"""Parameter-shift derivatives of the FP64 oracle spread over the host's cores (test infrastructure).

Each derivative needs the circuit evaluated twice from the shifted gate on; the state before that
gate is shared, so the circuit is walked once here and every (prefix state, shifted suffix) job goes
to a process pool. The pool uses the "spawn" start method: a process forked from a parent that has
already used CUDA can hang, and spawned workers import only numpy and the oracle.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os

import numpy as np

import oracle


def _shift_job(args):
    gates, which, n, params, inputs, grad_out, pre = args
    g = gates[which]
    vals = []
    for delta in (math.pi / 2, -math.pi / 2):
        params2 = np.concatenate([params, [0.0]])
        inputs2 = np.array(inputs, copy=True)
        if g[3] >= 0:
            params2[-1] = params[g[3]] + delta
            gs = (g[0], g[1], g[2], len(params2) - 1)
        else:
            col = -2 - g[3]
            inputs2 = np.concatenate([inputs2, inputs2[:, col:col + 1] + delta], axis=1)
            gs = (g[0], g[1], g[2], -2 - (inputs2.shape[1] - 1))
        psi = oracle.simulate_strided([gs] + list(gates[which + 1:]), n, params2, inputs2, init=pre)
        vals.append(np.sum(grad_out * oracle.expval_z(psi, n), axis=1))
    return which, (vals[0] - vals[1]) / 2


def shift_derivatives(gates, n, params, inputs, grad_out, which, processes=None):
    """{gate index: per-sample derivative (B,)} of sum(g * z) w.r.t. the angle of each listed gate
    occurrence (the exact +-pi/2 rule), evaluated in parallel."""
    gates = [tuple(g) for g in gates]
    params = np.asarray(params, dtype=np.float64)
    inputs = np.atleast_2d(np.asarray(inputs, dtype=np.float64))
    grad_out = np.atleast_2d(np.asarray(grad_out, dtype=np.float64))
    order = sorted(set(int(w) for w in which))
    jobs, at, psi = [], 0, None
    for w in order:                     # one walk: the state before each listed gate
        psi = oracle.simulate_strided(gates[at:w], n, params, inputs, init=psi)
        at = w
        jobs.append((gates, w, n, params, inputs, grad_out, psi.copy()))
    procs = processes or min(len(jobs), os.cpu_count() or 1)
    if procs <= 1:
        return dict(_shift_job(j) for j in jobs)
    with mp.get_context("spawn").Pool(procs) as pool:
        return dict(pool.map(_shift_job, jobs, chunksize=1))
