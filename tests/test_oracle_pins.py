"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a transposed matrix, a wrong sign, the
Kronecker factors in the wrong order, a dropped term in the measurement) makes it fail; the
``test_planted_*`` cases plant such slips in the oracle (monkeypatched, CPU only) and check that.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
import workloads as W
from oracle import gates as OG
from oracle.bitsim import simulate_bits, expval_z_bits

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ANGLES = [0.0, 0.3, 1.0, math.pi / 2, 2.5, math.pi, 4.0, 2 * math.pi - 0.1]


# ---------------------------------------------------------------- gate algebra
@pytest.mark.parametrize("theta", ANGLES)
def test_rotations_equal_matrix_exponential(theta):
    # R_P(theta) = exp(-i theta P / 2), computed by scipy's Pade expm, independent of Eq. 1
    for fn, P in ((OG.rx, OG.PX), (OG.ry, OG.PY), (OG.rz, OG.PZ)):
        np.testing.assert_allclose(fn(theta), expm(-0.5j * theta * P), atol=1e-14)


def test_fixed_gates_and_unitarity():
    np.testing.assert_allclose(OG.hadamard() @ OG.hadamard(), np.eye(2), atol=1e-15)
    np.testing.assert_allclose(OG.hadamard() * math.sqrt(2), [[1, 1], [1, -1]], atol=1e-15)
    np.testing.assert_allclose(OG.pauli_x(), [[0, 1], [1, 0]])
    for th in ANGLES:
        for fn in (OG.rx, OG.ry, OG.rz):
            U = fn(th)
            np.testing.assert_allclose(U.conj().T @ U, np.eye(2), atol=1e-15)


def test_rz_phase_convention():
    # RZ(theta) = diag(e^{-i theta/2}, e^{+i theta/2}), not diag(1, e^{i theta})
    th = 0.7
    np.testing.assert_allclose(OG.rz(th), np.diag([np.exp(-0.35j), np.exp(0.35j)]), atol=1e-15)


def test_expanded_gates_unitary():
    rng = np.random.default_rng(0)
    for W_ in (2, 3, 4):
        for q in range(W_):
            U = OG.expand_1q(OG.ry(rng.uniform(0, 6)), q, W_)
            np.testing.assert_allclose(U.conj().T @ U, np.eye(2 ** W_), atol=1e-14)
        for c in range(W_):
            for t in range(W_):
                if c != t:
                    U = OG.expand_controlled(c, t, OG.PX, W_)
                    np.testing.assert_allclose(U @ U, np.eye(2 ** W_), atol=0)
                    # a permutation matrix
                    assert np.all((U == 0) | (U == 1)) and np.all(U.sum(0) == 1)


# ---------------------------------------------------------------- layout (paper's worked examples)
def _read_examples():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_examples.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _x_gates_for_pattern(pattern):
    return [W.gate(W.X, (q,)) for q, ch in enumerate(pattern) if ch == "1"]


def test_paper_worked_examples():
    rows = _read_examples()
    assert len(rows) == 4
    for kind, n, pattern, expected, _cite in rows:
        n = int(n)
        if kind == "basis":
            psi = oracle.simulate_kron(_x_gates_for_pattern(pattern), n, [], np.zeros((1, 0)))[0]
            assert np.argmax(np.abs(psi)) == int(expected) and abs(psi[int(expected)]) == 1.0
        elif kind == "tensor":
            psi = oracle.simulate_kron(_x_gates_for_pattern(pattern), n, [], np.zeros((1, 0)))[0]
            pos = tuple(int(v) for v in expected.split(","))
            assert psi.reshape((2,) * n)[pos] == 1.0
        elif kind == "reshape":
            group = [int(v) for v in pattern.split(",")]
            shape = tuple(int(v) for v in expected.split(","))
            _check_reshape_example(n, group, shape)
        else:
            raise AssertionError(kind)


def _check_reshape_example(n, group, shape):
    """Sec. "Circuit Splitting": a sub-circuit on ``group`` is applied by viewing the state as
    (prod d_rest, prod d_group) and multiplying over the last axis; the result must equal the
    Kronecker oracle's sequential application of the same gates."""
    rng = np.random.default_rng(5)
    a, b = group
    sub = [W.gate(W.RY, (a,), param=0), W.gate(W.CNOT, (b,), (a,)), W.gate(W.RZ, (b,), param=1)]
    params = rng.uniform(0, 2 * math.pi, 2)
    init = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    init /= np.linalg.norm(init)
    want = oracle.simulate_kron(sub, n, params, np.zeros((1, 0)), init=init[None])[0]
    # group unitary on the two group qubits (local order a, b), as a 4x4 dense matrix
    U = np.eye(4, dtype=complex)
    local = [W.gate(W.RY, (0,), param=0), W.gate(W.CNOT, (1,), (0,)), W.gate(W.RZ, (1,), param=1)]
    for g in local:
        U = OG.full_gate_matrix(g, 2, params, None) @ U
    rest = [q for q in range(n) if q not in group]
    t = init.reshape((2,) * n).transpose(rest + group)
    mat = t.reshape(shape)
    assert mat.shape == shape
    out = (mat @ U.T).reshape((2,) * n)
    inv = np.argsort(rest + group)
    got = out.transpose(inv).reshape(-1)
    np.testing.assert_allclose(got, want, atol=1e-14)
    # batched form (b*d0*d3*d4, d1*d2)
    batch = np.stack([init, init.conj()])
    tb = batch.reshape((2,) + (2,) * n).transpose([0] + [1 + q for q in rest + group])
    assert tb.reshape(2 * shape[0], shape[1]).shape == (2 * shape[0], shape[1])


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_x_on_qubit_lands_at_msb0_index(n):
    for q in range(n):
        psi = oracle.simulate_kron([W.gate(W.X, (q,))], n, [], np.zeros((1, 0)))[0]
        assert psi[1 << (n - 1 - q)] == 1.0 and np.sum(np.abs(psi)) == 1.0


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 3, 6])
def test_hadamard_all_uniform(n):
    psi = oracle.simulate_kron([W.gate(W.H, (q,)) for q in range(n)], n, [], np.zeros((1, 0)))
    np.testing.assert_allclose(psi[0], np.full(2 ** n, 2 ** (-n / 2)), atol=1e-15)
    np.testing.assert_allclose(oracle.expval_z(psi, n), 0.0, atol=1e-15)


@pytest.mark.parametrize("n", [2, 4, 7])
def test_ghz(n):
    gates = [W.gate(W.H, (0,))] + [W.gate(W.CNOT, (q + 1,), (q,)) for q in range(n - 1)]
    for sim in (oracle.simulate_kron, oracle.simulate_strided):
        psi = sim(gates, n, [], np.zeros((1, 0)))
        np.testing.assert_allclose(oracle.expval_z(psi, n), 0.0, atol=1e-15)
        for i in range(n):
            for j in range(n):
                np.testing.assert_allclose(oracle.expval_zz(psi, n, i, j), 1.0, atol=1e-14)
        assert abs(psi[0, 0] - 2 ** -0.5) < 1e-15 and abs(psi[0, -1] - 2 ** -0.5) < 1e-15


def test_rx_chain_cosine_sum():
    rng = np.random.default_rng(1)
    for n, q in ((1, 0), (3, 1), (5, 4)):
        th = rng.uniform(0, 2 * math.pi, 7)
        gates = [W.gate(W.RX, (q,), param=k) for k in range(7)]
        for sim in (oracle.simulate_kron, oracle.simulate_strided):
            z = oracle.expval_z(sim(gates, n, th, np.zeros((1, 0))), n)[0]
            assert abs(z[q] - math.cos(th.sum())) < 1e-13
            for other in range(n):
                if other != q:
                    assert abs(z[other] - 1.0) < 1e-14


def test_product_state_closed_forms():
    rng = np.random.default_rng(2)
    n = 5
    x = rng.uniform(0, math.pi, (3, n))
    y = rng.uniform(0, 2 * math.pi, n)
    zang = rng.uniform(0, 2 * math.pi, n)
    gates = [W.gate(W.RX, (q,), param=W.input_param(q)) for q in range(n)]
    gates += [W.gate(W.RY, (q,), param=q) for q in range(n)]
    gates += [W.gate(W.RZ, (q,), param=n + q) for q in range(n)]
    params = np.concatenate([y, zang])
    for sim in (oracle.simulate_kron, oracle.simulate_strided):
        z = oracle.expval_z(sim(gates, n, params, x), n)
        np.testing.assert_allclose(z, np.cos(x) * np.cos(y)[None, :], atol=1e-13)
    # closed-form gradients of L = sum g z: dz_q/dy_q = -cos x sin y; dz_q/dx_q = -sin x cos y
    g = rng.uniform(-1, 1, (3, n))
    dp, di = oracle.grad_param_shift(gates, n, params, x, g)
    np.testing.assert_allclose(dp[:n], np.sum(-g * np.cos(x) * np.sin(y)[None, :], axis=0), atol=1e-12)
    np.testing.assert_allclose(dp[n:], 0.0, atol=1e-12)       # RZ after RY: no effect on <Z>
    np.testing.assert_allclose(di, -g * np.sin(x) * np.cos(y)[None, :], atol=1e-12)


def test_single_axis_rotations():
    for kind, expect in ((W.RX, math.cos), (W.RY, math.cos)):
        for th in ANGLES:
            z = oracle.forward_z([W.gate(kind, (0,), param=0)], 1, [th], np.zeros((1, 0)))[0, 0]
            assert abs(z - expect(th)) < 1e-14
    for th in ANGLES:     # RZ on |0> or after H leaves <Z> unchanged
        z = oracle.forward_z([W.gate(W.H, (0,)), W.gate(W.RZ, (0,), param=0)], 1, [th], np.zeros((1, 0)))
        assert abs(z[0, 0]) < 1e-15


@pytest.mark.parametrize("n", [3, 4, 6])
def test_cnot_ring_on_basis_states_is_bit_permutation(n):
    ring = [W.gate(W.CNOT, ((q + 1) % n,), (q,)) for q in range(n)]
    for x in range(2 ** n):
        bits = [(x >> (n - 1 - q)) & 1 for q in range(n)]
        prep = [W.gate(W.X, (q,)) for q in range(n) if bits[q]]
        b = list(bits)
        for q in range(n):               # classical simulation of the ring
            b[(q + 1) % n] ^= b[q]
        for sim in (oracle.simulate_kron, oracle.simulate_strided):
            z = oracle.expval_z(sim(prep + ring, n, [], np.zeros((1, 0))), n)[0]
            np.testing.assert_array_equal(z, [1.0 - 2.0 * v for v in b])


def test_cz_ladder_phases():
    n = 4
    gates = [W.gate(W.H, (q,)) for q in range(n)] + [W.gate(W.CZ, (q + 1,), (q,)) for q in range(n - 1)]
    psi = oracle.simulate_kron(gates, n, [], np.zeros((1, 0)))[0]
    for x in range(2 ** n):
        bits = [(x >> (n - 1 - q)) & 1 for q in range(n)]
        sign = (-1) ** sum(bits[q] * bits[q + 1] for q in range(n - 1))
        assert abs(psi[x] - sign * 0.25) < 1e-15


# ---------------------------------------------------------------- composition / brute force
def _random_circuit(rng, n, n_gates, n_params, n_inputs):
    gates = []
    for _ in range(n_gates):
        k = int(rng.integers(0, 7))
        if k in (W.RX, W.RY, W.RZ):
            q = int(rng.integers(0, n))
            p = int(rng.integers(0, n_params)) if rng.uniform() < 0.7 or n_inputs == 0 \
                else W.input_param(int(rng.integers(0, n_inputs)))
            gates.append(W.gate(k, (q,), param=p))
        elif k in (W.H, W.X):
            gates.append(W.gate(k, (int(rng.integers(0, n)),)))
        else:
            if n < 2:
                continue
            c, t = rng.choice(n, 2, replace=False)
            gates.append(W.gate(k, (int(t),), (int(c),)))
    return gates


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_brute_force_composition(n):
    rng = np.random.default_rng(10 + n)
    gates = _random_circuit(rng, n, 25, 6, 2)
    params = rng.uniform(0, 2 * math.pi, 6)
    inputs = rng.uniform(0, math.pi, (3, 2))
    psi = oracle.simulate_kron(gates, n, params, inputs)
    for b in range(3):
        U = np.eye(2 ** n, dtype=complex)
        state = np.zeros(2 ** n, dtype=complex); state[0] = 1
        for g in gates:
            G = OG.full_gate_matrix(g, n, params, inputs[b])
            U = G @ U
            state = G @ state
            assert abs(np.linalg.norm(state) - 1) < 1e-14
        np.testing.assert_allclose(U.conj().T @ U, np.eye(2 ** n), atol=1e-13)
        e0 = np.zeros(2 ** n); e0[0] = 1
        np.testing.assert_allclose(U @ e0, psi[b], atol=1e-13)
        bs = np.array(simulate_bits(gates, n, params, inputs[b]))
        np.testing.assert_allclose(bs, psi[b], atol=1e-13)
        np.testing.assert_allclose(expval_z_bits(list(bs), n), oracle.expval_z(psi[b:b + 1], n)[0], atol=1e-13)


@pytest.mark.parametrize("n", [2, 5, 8, 10])
def test_kron_equals_strided(n):
    rng = np.random.default_rng(20 + n)
    gates = _random_circuit(rng, n, 40, 8, 3)
    params = rng.uniform(0, 2 * math.pi, 8)
    inputs = rng.uniform(0, math.pi, (2, 3))
    init = rng.normal(size=(2, 2 ** n)) + 1j * rng.normal(size=(2, 2 ** n))
    init /= np.linalg.norm(init, axis=1, keepdims=True)
    a = oracle.simulate_kron(gates, n, params, inputs, init=init)
    b = oracle.simulate_strided(gates, n, params, inputs, init=init)
    np.testing.assert_allclose(a, b, atol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-13)


def test_golden_c1_regression():
    wl = W.config(1)
    z = oracle.forward_z(wl.gates, wl.n, wl.params, wl.inputs)
    want = np.loadtxt(os.path.join(GOLDEN, "c1_z.txt"))
    np.testing.assert_allclose(z, want, atol=1e-14)
    lines = [l for l in open(os.path.join(GOLDEN, "c1_grad.txt")) if not l.startswith("#")]
    rows = [np.array([float(v) for v in l.split()]) for l in lines]
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out)
    np.testing.assert_allclose(dp, rows[0], atol=1e-13)
    np.testing.assert_allclose(di, np.stack(rows[1:]), atol=1e-13)


# ---------------------------------------------------------------- gradients
def test_param_shift_equals_finite_difference():
    wl = W.config(1)
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out)
    fp, fi = oracle.grad_finite_diff(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out, h=1e-4)
    np.testing.assert_allclose(dp, fp, atol=1e-8)
    np.testing.assert_allclose(di, fi, atol=1e-8)


def test_param_shift_with_shared_parameter_and_strided():
    rng = np.random.default_rng(3)
    n = 4
    gates = _random_circuit(rng, n, 30, 3, 2)        # only 3 params: heavy reuse
    params = rng.uniform(0, 2 * math.pi, 3)
    inputs = rng.uniform(0, math.pi, (2, 2))
    g = rng.uniform(-1, 1, (2, n))
    dk = oracle.grad_param_shift(gates, n, params, inputs, g, method="kron")
    ds = oracle.grad_param_shift(gates, n, params, inputs, g, method="strided")
    fd = oracle.grad_finite_diff(gates, n, params, inputs, g, h=1e-4)
    for a, b in zip(dk, ds):
        np.testing.assert_allclose(a, b, atol=1e-13)
    for a, b in zip(dk, fd):
        np.testing.assert_allclose(a, b, atol=1e-8)


# ---------------------------------------------------------------- adjoint sweep (oracle.grad_adjoint)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_equals_param_shift_kron(seed):
    # every gate type, shared parameters, input columns and (seed 1) a random initial state, against
    # the exact shift rule evaluated on the dense Kronecker oracle (no code in common with the sweep)
    rng = np.random.default_rng(40 + seed)
    n, B = 5, 3
    gates = _random_circuit(rng, n, 45, 4, 2)
    params = rng.uniform(0, 2 * math.pi, 4)
    inputs = rng.uniform(0, math.pi, (B, 2))
    g = rng.uniform(-1, 1, (B, n))
    init = None
    if seed == 1:
        init = rng.normal(size=(B, 2 ** n)) + 1j * rng.normal(size=(B, 2 ** n))
        init /= np.linalg.norm(init, axis=1, keepdims=True)
    da, ia = oracle.grad_adjoint(gates, n, params, inputs, g, init=init)
    dk, ik = oracle.grad_param_shift(gates, n, params, inputs, g, method="kron", init=init)
    np.testing.assert_allclose(da, dk, atol=1e-12)
    np.testing.assert_allclose(ia, ik, atol=1e-12)


def test_adjoint_product_state_closed_form():
    # RX(x_q) then RY(t_q) on every qubit, no entanglers: <Z_q> = cos x_q cos t_q, so
    # dL/dt_q = -g_q cos x_q sin t_q and dL/dx_q = -g_q sin x_q cos t_q
    rng = np.random.default_rng(7)
    n, B = 4, 2
    gates = [W.gate(W.RX, (q,), param=W.input_param(q)) for q in range(n)]
    gates += [W.gate(W.RY, (q,), param=q) for q in range(n)]
    t = rng.uniform(0, 2 * math.pi, n)
    x = rng.uniform(0, math.pi, (B, n))
    g = rng.uniform(-1, 1, (B, n))
    dp, di = oracle.grad_adjoint(gates, n, t, x, g)
    np.testing.assert_allclose(dp, (-g * np.cos(x) * np.sin(t)).sum(axis=0), atol=1e-14)
    np.testing.assert_allclose(di, -g * np.sin(x) * np.cos(t), atol=1e-14)


def _adjoint_pins_pass():
    try:
        test_adjoint_equals_param_shift_kron(0)
        test_adjoint_product_state_closed_form()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mistake", ["no_dagger", "real_part", "lambda_not_uncomputed", "pauli_wrong_axis"])
def test_planted_adjoint_mistakes_are_caught(monkeypatch, mistake):
    import oracle.adjoint as A
    assert _adjoint_pins_pass()
    if mistake == "no_dagger":
        orig = A._gate_dagger
        monkeypatch.setattr(A, "_gate_dagger", lambda g, p, x, b: np.conj(np.swapaxes(orig(g, p, x, b), -1, -2)))
    elif mistake == "real_part":
        monkeypatch.setattr(A, "np", type("npx", (), {**{k: getattr(np, k) for k in dir(np) if not k.startswith("__")},
                                                    "imag": staticmethod(np.real)}))
    elif mistake == "lambda_not_uncomputed":
        orig1 = A._apply_1q
        monkeypatch.setattr(A, "_apply_1q", lambda psi, n, w, G: psi if psi is A._LAST_LAM else orig1(psi, n, w, G))
        orig_lo = A._loss_observable

        def keep(psi, n, g):
            lam = orig_lo(psi, n, g)
            A._LAST_LAM = lam
            return lam
        monkeypatch.setattr(A, "_LAST_LAM", None, raising=False)
        monkeypatch.setattr(A, "_loss_observable", keep)
    elif mistake == "pauli_wrong_axis":
        monkeypatch.setattr(A, "_PAULI", {W.RX: OG.PY, W.RY: OG.PX, W.RZ: OG.PZ})
    assert not _adjoint_pins_pass(), f"planted adjoint mistake {mistake} was not caught by any pin"


# ---------------------------------------------------------------- planted mistakes
def _pins_pass():
    try:
        for th in ANGLES:
            test_rotations_equal_matrix_exponential(th)
        test_paper_worked_examples()
        for n in (1, 3, 6):
            test_hadamard_all_uniform(n)
        test_rx_chain_cosine_sum()
        test_product_state_closed_forms()
        test_cnot_ring_on_basis_states_is_bit_permutation(3)
        test_brute_force_composition(3)
        test_kron_equals_strided(5)
    except AssertionError:
        return False
    return True


def test_pins_pass_unmodified():
    assert _pins_pass()


@pytest.mark.parametrize("mistake", ["ry_transposed", "rz_sign", "kron_order", "measure_lsb",
                                     "cnot_swapped", "rx_dropped_term"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    import oracle.gates as g
    import oracle.measure as m
    if mistake == "ry_transposed":
        orig = g.ry
        monkeypatch.setattr(g, "ry", lambda th: orig(th).T)
    elif mistake == "rz_sign":
        orig = g.rz
        monkeypatch.setattr(g, "rz", lambda th: orig(-th))
    elif mistake == "rx_dropped_term":
        monkeypatch.setattr(g, "rx", lambda th: g.I2 * np.cos(th / 2) + 0 * g.PX)
    elif mistake == "kron_order":
        monkeypatch.setattr(g, "expand_1q", lambda G, w, W_: np.kron(np.kron(
            np.eye(2 ** (W_ - 1 - w), dtype=complex), G), np.eye(2 ** w, dtype=complex)))
    elif mistake == "measure_lsb":
        def bad(psi, n):
            psi = np.atleast_2d(psi)
            prob = np.abs(psi) ** 2
            x = np.arange(2 ** n)
            return np.stack([prob @ (1.0 - 2.0 * ((x >> i) & 1)) for i in range(n)], axis=1)
        monkeypatch.setattr(m, "expval_z", bad)
        monkeypatch.setattr(oracle, "expval_z", bad)
        import oracle.grad as gr
        monkeypatch.setattr(gr, "expval_z", bad)
    elif mistake == "cnot_swapped":
        orig = g.expand_controlled
        monkeypatch.setattr(g, "expand_controlled", lambda c, t, U, W_: orig(t, c, U, W_))
    assert not _pins_pass(), f"planted mistake {mistake} was not caught by any pin"


# ---------------------------------------------------------------- quantum weight remapping (Sec. "Additional Optimizations")
def test_remap_range_and_fixed_points():
    w = np.linspace(-6, 6, 41)
    a = oracle.remap(w)
    assert np.all(np.abs(a) < math.pi) and np.all(np.diff(a) > 0)       # into (-pi, pi), monotone
    np.testing.assert_allclose(oracle.remap(-w), -a, atol=0)              # odd
    np.testing.assert_allclose(oracle.remap(np.arctanh([0.5, -0.25])), [math.pi / 2, -math.pi / 4], atol=1e-15)


@pytest.mark.parametrize("w", [-1.7, -0.4, 0.0, 0.3, 1.1, 2.6])
def test_remap_single_rx_closed_form(w):
    # RX(pi tanh w)|0>: <Z> = cos(pi tanh w), d<Z>/dw = -sin(pi tanh w) * pi (1 - tanh^2 w)
    gates = [(W.RX, (0, -1), (-1, -1), 0)]
    z = oracle.forward_z_remapped(gates, 1, [w], np.zeros((1, 0)))
    np.testing.assert_allclose(z[0, 0], math.cos(math.pi * math.tanh(w)), atol=1e-14)
    dp, _ = oracle.grad_remapped(gates, 1, [w], np.zeros((1, 0)), np.ones((1, 1)))
    t = math.tanh(w)
    np.testing.assert_allclose(dp[0], -math.sin(math.pi * t) * math.pi * (1 - t * t), atol=1e-13)


def test_remap_chain_rule_equals_finite_difference_on_raw_weights():
    wl = W.config(1, n=3, batch=2, layers=1)
    w = wl.params - math.pi          # spread over both signs of tanh
    dp, di = oracle.grad_remapped(wl.gates, wl.n, w, wl.inputs, wl.grad_out)
    h = 1e-5
    for p in range(len(w)):
        wp = w.copy(); wp[p] += h
        wm = w.copy(); wm[p] -= h
        lp = oracle.loss(oracle.forward_z_remapped(wl.gates, wl.n, wp, wl.inputs), wl.grad_out)
        lm = oracle.loss(oracle.forward_z_remapped(wl.gates, wl.n, wm, wl.inputs), wl.grad_out)
        assert abs(dp[p] - (lp - lm) / (2 * h)) < 1e-8
    # inputs are not remapped: their gradient is the plain one
    _, di_plain = oracle.grad_param_shift(wl.gates, wl.n, oracle.remap(w), wl.inputs, wl.grad_out)
    np.testing.assert_allclose(di, di_plain, atol=0)


def test_planted_remap_slope_mistake_is_caught(monkeypatch):
    from oracle import remapping as R
    monkeypatch.setattr(R, "remap_slope", lambda w: np.pi * (1.0 - np.tanh(np.asarray(w, dtype=np.float64))))
    with pytest.raises(AssertionError):
        test_remap_single_rx_closed_form(1.1)


# ---------------------------------------------------------------- parallel shift-rule helper of the GPU tests
def test_parallel_shift_derivatives_equal_serial_shift_rule():
    from oracle_pool import shift_derivatives
    wl = W.config(3, n=6, batch=2, layers=2)          # every parameter and input column used once
    which = [i for i, g in enumerate(wl.gates) if g[3] != -1]
    d = shift_derivatives(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out, which, processes=2)
    dp, di = oracle.grad_param_shift(wl.gates, wl.n, wl.params, wl.inputs, wl.grad_out, method="kron")
    for i, v in d.items():
        p = wl.gates[i][3]
        if p >= 0:
            assert abs(v.sum() - dp[p]) < 1e-12
        else:
            np.testing.assert_allclose(v, di[:, -2 - p], atol=1e-12)
