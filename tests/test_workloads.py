"""Seeded workload generator: published splitmix64 vectors, determinism and the config shapes."""
import math

import numpy as np

import workloads as W


def test_splitmix64_published_vector():
    # splitmix64 seeded with 0 (Steele et al.; the reference C code in xoshiro's seeding notes)
    r = W.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4


def test_uniform_range_and_determinism():
    a = W.SplitMix64(7).uniforms(1000)
    b = W.SplitMix64(7).uniforms(1000)
    assert np.array_equal(a, b) and a.min() >= 0.0 and a.max() < 1.0


def test_config_counts():
    expect = {1: (4, 8, 28, 16), 2: (12, 1024, 228, 144), 3: (20, 64, 620, 400), 5: (30, 1, 750, 480)}
    for c, (n, B, G, P) in expect.items():
        wl = W.config(c)
        assert (wl.n, wl.batch, len(wl.gates), wl.n_params) == (n, B, G, P)
        assert wl.inputs.shape == (B, n) and wl.grad_out.shape == (B, n)
        assert np.all((wl.inputs >= 0) & (wl.inputs < math.pi))
        assert np.all((wl.params >= 0) & (wl.params < 2 * math.pi))
        assert np.all((wl.grad_out >= -1) & (wl.grad_out < 1))


def test_ring_structure():
    g = W.ring_ansatz(3, 1)
    assert g[:3] == [W.gate(W.RX, (q,), param=-2 - q) for q in range(3)]
    assert [x[0] for x in g[3:9]] == [W.RY] * 3 + [W.RZ] * 3
    assert g[9:] == [W.gate(W.CNOT, (1,), (0,)), W.gate(W.CNOT, (2,), (1,)), W.gate(W.CNOT, (0,), (2,))]


def test_multi_circuit_config():
    m = W.multi_circuit_config()
    assert len(m) == 256
    assert all(8 <= w.n <= 22 and 4 <= w.meta["depth"] <= 16 and w.batch == 4 for w in m)
    for w in m[:10]:
        assert len(w.gates) == w.n + w.meta["depth"] * (3 * w.n - 1)
        assert w.n_params == 2 * w.n * w.meta["depth"]
    again = W.multi_circuit_config()
    assert all(np.array_equal(a.params, b.params) and a.n == b.n for a, b in zip(m, again))
