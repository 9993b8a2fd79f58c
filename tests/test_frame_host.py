"""Pauli-frame bookkeeping of pauli_frame plans, checked on the host with the library's own frame walk
(the code the device walk runs): a kernel that applies every rotation in the tangent form only, with the
coefficient sign sigma the walk returns (sigma * tan, or -sigma * cot for the cotangent form), gives the
true state as scale * F * (kernel state), <Z_q> with the sign F gives Z_q, and adjoint gradients
sigma * bs^2 * Im<lambda|P|psi> equal to central differences. Dense 4-qubit matrices; no GPU needed."""
import ctypes

import numpy as np
import pytest

import workloads as W

N = 4
D = 2 ** N
I2 = np.eye(2)
PX = np.array([[0, 1], [1, 0]], complex)
PY = np.array([[0, -1j], [1j, 0]])
PZ = np.diag([1.0, -1.0]).astype(complex)
PAULI = {W.RX: PX, W.RY: PY, W.RZ: PZ}
HAD = np.array([[1, 1], [1, -1]]) / np.sqrt(2)


@pytest.fixture(scope="module")
def lib():
    from paper_2404_09213_gb300 import build
    build.build()
    from paper_2404_09213_gb300 import _lib
    return _lib.lib()


def op1(u, q):
    m = np.array([[1.0]])
    for j in range(N):
        m = np.kron(m, u if j == q else I2)
    return m


def two(kind, c, t):
    m = np.zeros((D, D), complex)
    for i in range(D):
        bc, bt = (i >> (N - 1 - c)) & 1, (i >> (N - 1 - t)) & 1
        if kind == W.CNOT:
            m[i ^ (bc << (N - 1 - t)), i] = 1
        else:
            m[i, i] = -1 if bc and bt else 1
    return m


def gate_matrix(g, theta=None):
    kind, q, c = g[0], g[1][0], g[2][0]
    if kind in PAULI:
        return op1(np.cos(theta / 2) * I2 - 1j * np.sin(theta / 2) * PAULI[kind], q)
    if kind == W.H:
        return op1(HAD, q)
    if kind == W.X:
        return op1(PX, q)
    return two(kind, c, q)


def frame_matrix(x, z, k):
    m = np.array([[1.0]], complex)
    for q in range(N):
        b = np.eye(2, dtype=complex)
        if (z >> q) & 1:
            b = PZ @ b
        if (x >> q) & 1:
            b = PX @ b
        m = np.kron(m, b)
    return (1j ** k) * m


def walk(lib, gates, cot):
    n = len(gates)
    arr = lambda v, t: (t * max(n, 1))(*v)
    types = arr([g[0] for g in gates], ctypes.c_int32)
    q0 = arr([g[1][0] for g in gates], ctypes.c_int32)
    q1 = arr([g[2][0] for g in gates], ctypes.c_int32)
    cf = arr([int(c) for c in cot], ctypes.c_uint8)
    sig = (ctypes.c_int8 * max(n, 1))()
    x, z, k = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int32()
    assert lib.qsim_frame_walk_host(types, q0, q1, cf, n, sig, ctypes.byref(x), ctypes.byref(z), ctypes.byref(k)) == 0
    return [int(s) for s in sig[:n]], x.value, z.value, k.value


def random_gates(rng, count, n_params):
    out = []
    for _ in range(count):
        kind = int(rng.integers(0, 7))
        if kind in PAULI:
            out.append(W.gate(kind, (int(rng.integers(N)),), param=int(rng.integers(n_params))))
        elif kind in (W.H, W.X):
            out.append(W.gate(kind, (int(rng.integers(N)),)))
        else:
            c, t = rng.choice(N, 2, replace=False)
            out.append(W.gate(kind, (int(t),), (int(c),)))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_tangent_form_kernel_with_frame_reproduces_the_circuit(lib, seed):
    rng = np.random.default_rng(seed)
    n_params = 5
    gates = random_gates(rng, 24, n_params)
    theta = rng.uniform(-7, 7, n_params)
    gvec = rng.uniform(-1, 1, N)
    half = [theta[g[3]] / 2 if g[0] in PAULI else 0.0 for g in gates]
    cot = [g[0] in PAULI and abs(np.sin(h)) > abs(np.cos(h)) for g, h in zip(gates, half)]
    sigma, x, z, k = walk(lib, gates, cot)
    # forward, tangent form only
    S = np.zeros(D, complex)
    S[0] = 1
    scale = 1.0
    coef = []
    for g, h, ct, sg in zip(gates, half, cot, sigma):
        if g[0] in PAULI:
            s, c = np.sin(h), np.cos(h)
            cj = -sg * c / s if ct else sg * s / c
            scale *= s if ct else c
            coef.append(cj)
            S = op1(I2 - 1j * cj * PAULI[g[0]], g[1][0]) @ S
        else:
            coef.append(None)
            S = gate_matrix(g) @ S
    exact = np.zeros(D, complex)
    exact[0] = 1
    for g in gates:
        exact = gate_matrix(g, theta[g[3]] if g[0] in PAULI else None) @ exact
    np.testing.assert_allclose(scale * frame_matrix(x, z, k) @ S, exact, atol=1e-12)
    S = scale * S
    zsign = [-1 if (x >> q) & 1 else 1 for q in range(N)]
    zq = [zsign[q] * np.vdot(S, op1(PZ, q) @ S).real for q in range(N)]
    np.testing.assert_allclose(zq, [np.vdot(exact, op1(PZ, q) @ exact).real for q in range(N)], atol=1e-12)
    # adjoint backward in the stored representation
    lam = sum(gvec[q] * zsign[q] * (op1(PZ, q) @ S) for q in range(N))
    psi, bs, grad = S.copy(), 1.0, np.zeros(n_params)
    for g, h, ct, sg, cj in reversed(list(zip(gates, half, cot, sigma, coef))):
        if g[0] in PAULI:
            P = op1(PAULI[g[0]], g[1][0])
            grad[g[3]] += sg * bs * bs * np.vdot(lam, P @ psi).imag
            U = op1(I2 + 1j * cj * PAULI[g[0]], g[1][0])
            psi, lam = U @ psi, U @ lam
            bs *= np.sin(h) if ct else np.cos(h)
        else:
            G = gate_matrix(g).conj().T
            psi, lam = G @ psi, G @ lam
    start = np.zeros(D, complex)
    start[0] = 1
    np.testing.assert_allclose(bs * psi, start, atol=1e-12)

    def loss(th):
        v = np.zeros(D, complex)
        v[0] = 1
        for g in gates:
            v = gate_matrix(g, th[g[3]] if g[0] in PAULI else None) @ v
        return sum(gvec[q] * np.vdot(v, op1(PZ, q) @ v).real for q in range(N))
    for p in range(n_params):
        e = np.zeros(n_params)
        e[p] = 1e-5
        assert abs(grad[p] - (loss(theta + e) - loss(theta - e)) / 2e-5) < 1e-7, p


def test_frame_walk_rejects_null_arguments(lib):
    x, z, k = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int32()
    assert lib.qsim_frame_walk_host(None, None, None, None, 3, None, ctypes.byref(x), ctypes.byref(z),
                                    ctypes.byref(k)) != 0


def test_fixup_formula_applies_the_frame():
    # the returned-state fix-up: out[i] = i^k (-1)^popc(zi & (i ^ xi)) S[i ^ xi], with the qubit masks
    # bit-reversed into index bits (qubit q at index bit N - 1 - q)
    rng = np.random.default_rng(9)
    brev = lambda v: int(f"{v:064b}"[::-1], 2) >> (64 - N)
    for _ in range(50):
        x, z, k = int(rng.integers(D)), int(rng.integers(D)), int(rng.integers(4))
        S = rng.normal(size=D) + 1j * rng.normal(size=D)
        xi, zi = brev(x), brev(z)
        out = np.array([(1j ** k) * (-1) ** bin(zi & (i ^ xi)).count("1") * S[i ^ xi] for i in range(D)])
        np.testing.assert_allclose(out, frame_matrix(x, z, k) @ S, atol=1e-12)
