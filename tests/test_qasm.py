"""OpenQASM 2.0 import / export (host only): exact gate lists, angle expressions, register handling,
errors with line numbers, bit-exact round trips, and the same state as the source circuit."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def q():
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def g(kind, t, c=-1, p=-1):
    return (kind, (t, -1), (c, -1), p)


def test_basic_program(q):
    text = """OPENQASM 2.0;
include "qelib1.inc";
qreg q[3];
creg c[3];
h q[0];
cx q[0],q[1];
rx(pi/2) q[2];
ry(-0.25) q[1];
rz(2*pi/3) q[0];
cz q[2],q[0];
x q[1];
barrier q;
measure q -> c;
"""
    gates, params, n = q.parse_qasm(text)
    assert n == 3
    assert gates == [g(W.H, 0), g(W.CNOT, 1, 0), g(W.RX, 2, p=0), g(W.RY, 1, p=1), g(W.RZ, 0, p=2),
                     g(W.CZ, 0, 2), g(W.X, 1)]
    np.testing.assert_array_equal(params, [math.pi / 2, -0.25, 2 * math.pi / 3])


def test_registers_concatenate_and_broadcast(q):
    text = """OPENQASM 2.0; include "qelib1.inc";
qreg a[2]; qreg b[3];   // qubits a[0..1] = 0..1, b[0..2] = 2..4
h a;                     // broadcast over the register
cx a[1], b;              // one control, every target of b
cx a, b[0:0+0];
"""
    with pytest.raises(q.QsimError):
        q.parse_qasm(text)                       # slices are not OpenQASM 2
    text = text.replace("cx a, b[0:0+0];", "rz(-pi) b;\ncx a, a;")
    with pytest.raises(q.QsimError, match="same qubit"):
        q.parse_qasm(text)
    text = text.replace("cx a, a;", "id b[1];")
    gates, params, n = q.parse_qasm(text)
    assert n == 5
    assert gates == [g(W.H, 0), g(W.H, 1), g(W.CNOT, 2, 1), g(W.CNOT, 3, 1), g(W.CNOT, 4, 1),
                     g(W.RZ, 2, p=0), g(W.RZ, 3, p=1), g(W.RZ, 4, p=2)]
    np.testing.assert_array_equal(params, [-math.pi] * 3)


@pytest.mark.parametrize("expr,value", [("pi", math.pi), ("-pi/4", -math.pi / 4), ("(pi+1)/2", (math.pi + 1) / 2),
                                        ("1e-3", 1e-3), ("-(0.5)", -0.5), ("2*pi/3-1", 2 * math.pi / 3 - 1),
                                        (".5*-2", -1.0), ("3", 3.0)])
def test_angle_expressions(q, expr, value):
    _, params, _ = q.parse_qasm(f"OPENQASM 2.0; qreg q[1]; rx({expr}) q[0];")
    assert params[0] == value


@pytest.mark.parametrize("body,msg", [("u3(1,2,3) q[0];", "unsupported"), ("h r[0];", "unknown quantum register"),
                                      ("h q[4];", "out of range"), ("h q[0]", "expected ';'"),
                                      ("rx(theta) q[0];", "unknown symbol"), ("rx(1/0) q[0];", "division by zero"),
                                      ("h(1) q[0];", "takes no angle"), ("qreg q[2];", "declared twice")])
def test_errors_name_the_line(q, body, msg):
    text = "OPENQASM 2.0;\nqreg q[2];\n" + body + "\n"
    with pytest.raises(q.QsimError, match=msg) as e:
        q.parse_qasm(text)
    assert "line 3" in str(e.value)


def test_header_errors(q):
    with pytest.raises(q.QsimError, match="2.x"):
        q.parse_qasm("OPENQASM 3.0; qreg q[1];")
    with pytest.raises(q.QsimError, match="qelib1"):
        q.parse_qasm('OPENQASM 2.0; include "stdgates.inc"; qreg q[1];')
    with pytest.raises(q.QsimError, match="no quantum register"):
        q.parse_qasm("OPENQASM 2.0;")


def test_round_trip_is_bit_exact(q):
    rng = np.random.default_rng(3)
    text = "OPENQASM 2.0;\nqreg q[4];\n" + "".join(
        f"r{'xyz'[i % 3]}({rng.uniform(-7, 7)!r}) q[{i % 4}];\ncx q[{i % 4}],q[{(i + 1) % 4}];\n" for i in range(12))
    gates, params, n = q.parse_qasm(text)
    out = q.export_qasm(gates, n, params)
    gates2, params2, n2 = q.parse_qasm(out)
    assert (gates2, n2) == (gates, n)
    assert params2.tobytes() == params.tobytes()


def test_export_then_import_gives_the_same_state(q):
    wl = W.config(1, n=4, batch=2, layers=2)
    for b in range(2):
        text = q.export_qasm(wl.gates, wl.n, wl.params, wl.inputs[b])
        gates, params, n = q.parse_qasm(text)
        assert n == wl.n and len(gates) == len(wl.gates)
        psi = oracle.simulate_kron(wl.gates, wl.n, wl.params, wl.inputs[b:b + 1])
        psi2 = oracle.simulate_kron(gates, n, params, np.zeros((1, 0)))
        np.testing.assert_allclose(psi2, psi, atol=1e-13)


def test_export_errors(q):
    with pytest.raises(q.QsimError):
        q.export_qasm([g(W.RX, 0, p=0)], 1)                 # angle needed but no params
    with pytest.raises(q.QsimError):
        q.export_qasm([g(W.CNOT, 0, 0)], 2)                 # control == target
    with pytest.raises(q.QsimError):
        q.export_qasm([g(W.H, 3)], 2)                       # target out of range


def test_random_circuits_round_trip(q):
    # every gate kind, random qubits, angles of very different magnitudes, empty circuits: the parsed
    # list is the exported one and the angles come back as the same doubles
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(1, 9))
        gates, angles = [], []
        for _ in range(int(rng.integers(0, 40))):
            kind = int(rng.integers(0, 7))
            t = int(rng.integers(0, n))
            if kind in (W.CNOT, W.CZ):
                if n < 2:
                    continue
                c = int((t + rng.integers(1, n)) % n)
                gates.append(g(kind, t, c))
            elif kind in (W.RX, W.RY, W.RZ):
                gates.append(g(kind, t, p=len(angles)))
                angles.append(float(rng.choice([rng.normal(), rng.uniform(-1e6, 1e6), rng.uniform(-1e-9, 1e-9)])))
            else:
                gates.append(g(kind, t))
        text = q.export_qasm(gates, n, angles)
        g2, p2, n2 = q.parse_qasm(text)
        assert n2 == n and g2 == gates, trial
        assert p2.tobytes() == np.array(angles, dtype=np.float64).tobytes(), trial
