"""Host planner invariants (bit-exact): every gate emitted once, per-wire order kept, passes k-local,
register phases consistent, shared-memory layouts bijective, gather/scatter index maps equal to a
brute-force permutation of the 2^n indices."""
import itertools
import random

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def q():
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    return q


def random_circuit(rng, n, g, n_params=6, n_inputs=2):
    out = []
    for _ in range(g):
        k = rng.randrange(7)
        if k in (W.RX, W.RY, W.RZ):
            p = rng.randrange(n_params) if (rng.random() < 0.7 or n_inputs == 0) else W.input_param(rng.randrange(n_inputs))
            out.append(W.gate(k, (rng.randrange(n),), param=p))
        elif k in (W.H, W.X):
            out.append(W.gate(k, (rng.randrange(n),)))
        elif n >= 2:
            c, t = rng.sample(range(n), 2)
            out.append(W.gate(k, (t,), (c,)))
    return out


def gate_qubits(g):
    return [g[1][0]] + ([g[2][0]] if g[2][0] >= 0 else [])


CASES = [("ring20", W.ring_ansatz(20, 10), 20, {}), ("ring12", W.ring_ansatz(12, 6), 12, {}),
         ("ring30", W.ring_ansatz(30, 2), 30, {}), ("hea15", W.hea_cz_ansatz(15, 5), 15, {}),
         ("ring20k8", W.ring_ansatz(20, 3), 20, {"k": 8}), ("ring10c2", W.ring_ansatz(10, 3), 10, {"k": 6, "contiguous_bits": 2}),
         ("c128", W.ring_ansatz(16, 3), 16, {"dtype": "c128"}),
         ("ring20rot", W.ring_ansatz(20, 10), 20, {"rotate_low_bits": True}),
         ("ring30rot", W.ring_ansatz(30, 2), 30, {"rotate_low_bits": True, "k": 11}),
         ("hea15rot", W.hea_cz_ansatz(15, 5), 15, {"rotate_low_bits": True, "k": 10}),
         ("c128rot", W.ring_ansatz(16, 3), 16, {"dtype": "c128", "rotate_low_bits": True})]
_r = random.Random(7)
for i in range(12):
    n = _r.randint(1, 14)
    CASES.append((f"rand{i}", random_circuit(_r, n, _r.randint(0, 60)), n,
                  {"k": _r.randint(min(n, 6), 12), "rotate_low_bits": bool(i % 2)}))


@pytest.mark.parametrize("name,gates,n,kw", CASES, ids=[c[0] for c in CASES])
def test_schedule_invariants(q, name, gates, n, kw):
    p = q.Plan(gates, n, **kw)
    d = p.describe()
    k, R = d["k"], d["R"]
    # the product-state prefix (each qubit's single-qubit gates before its first two-qubit gate) runs
    # before every pass; the per-wire order check below also proves no prefix gate follows an entangler
    order = [g for pq in d["prefix"] for g in pq] + [g for ps in d["passes"] for g in ps["gates"]]
    # every gate exactly once
    assert sorted(order) == list(range(len(gates)))
    # per-wire order preserved across passes
    pos = {g: i for i, g in enumerate(order)}
    last = {}
    for gi, g in enumerate(gates):
        for w in gate_qubits(g):
            if w in last:
                assert pos[last[w]] < pos[gi], f"wire {w}: gate {gi} before {last[w]}"
            last[w] = gi
    check_layouts(d, n)
    for ps in d["passes"]:
        local = ps["local_qubits"]
        assert len(local) == k and len(set(local)) == k
        c = d["c"]
        assert ps["L"][:c] == list(range(c)), "low index bits of the read layout must be local (coalescing)"
        assert set(range(c)) <= set(ps["Lo"]), "low index bits of the written layout must be local"
        assert ps["Lo"][0] == 0, "bit 0 (the 16-byte pair) keeps its qubit"
        for g in ps["gates"]:
            assert set(gate_qubits(gates[g])) <= set(local)
        for ph_key, lay_key, RR in (("phases", "layouts", R), ("bwd_phases", "bwd_layouts", d["Rb"])):
            check_phases(gates, ps, ps[ph_key], ps[lay_key], k, RR, local)
        # gradient slots (backward ops): one per rotation, dense
        slots = sorted(op["gslot"] for ph in ps["bwd_phases"] for op in ph["ops"] if op["gslot"] >= 0)
        assert slots == list(range(ps["n_gslots"]))
        assert ps["n_gslots"] == sum(1 for g in ps["gates"] if gates[g][0] in (W.RX, W.RY, W.RZ))


def layout(ps, out):
    """qubit -> physical bit of the layout a pass reads (out=False) or writes (out=True)."""
    L, NL = (ps["Lo"], ps["nonlocal_o"]) if out else (ps["L"], ps["nonlocal"])
    m = {q_: b for q_, b in zip(ps["local_qubits"], L)}
    m.update({q_: b for q_, b in zip(ps["QN"], NL)})
    return m


def check_layouts(d, n):
    canon = {q_: n - 1 - q_ for q_ in range(n)}
    passes = d["passes"]
    for ps in passes:
        for out in (False, True):
            m = layout(ps, out)
            assert sorted(m) == list(range(n)) and sorted(m.values()) == list(range(n)), "a bijection"
    assert layout(passes[0], False) == canon, "the first pass reads the canonical layout"
    assert layout(passes[-1], True) == canon, "the last pass writes the canonical layout"
    for a, b in zip(passes, passes[1:]):
        assert layout(a, True) == layout(b, False), "a pass reads the layout its predecessor wrote"
    # every pass but the last writes exactly the addresses it reads (only qubits of its tile change
    # places), so those passes may update a buffer in place
    for ps in passes[:-1]:
        assert ps["nonlocal_o"] == ps["nonlocal"] and sorted(ps["Lo"]) == sorted(ps["L"])


RESCALE_EVERY, MAX_SCALED_PER_PASS = 48, 256


def check_rescale(gates, ps, phases):
    # unnormalised ops (rotations, Hadamards) between two rescale ops: exactly RESCALE_EVERY; after the
    # last one at most that many, and a rescale op is never the pass's last op
    ops = [op for ph in phases for op in ph["ops"]]
    scaled = [op["kind"] != "scale" and gates[op["gate"]][0] in (W.RX, W.RY, W.RZ, W.H) for op in ops]
    assert sum(scaled) <= MAX_SCALED_PER_PASS
    run = 0
    for op, sc in zip(ops, scaled):
        if op["kind"] == "scale":
            assert op["gate"] == -1 and op["gslot"] == -1
            assert run == RESCALE_EVERY, run
            run = 0
        run += sc
    assert run <= RESCALE_EVERY
    assert not ops or ops[-1]["kind"] != "scale"


def check_phases(gates, ps, phases, layouts, k, R, local):
    # phases: same gates, order per wire preserved, register bits hold the targets that need them
    check_rescale(gates, ps, phases)
    phases = [dict(ph, ops=[op for op in ph["ops"] if op["kind"] != "scale"]) for ph in phases]
    ph_order = [op["gate"] for ph in phases for op in ph["ops"]]
    assert sorted(ph_order) == sorted(ps["gates"])
    last_in_pass = {}
    ppos = {g: i for i, g in enumerate(ph_order)}
    for g in sorted(ps["gates"]):
        for w in gate_qubits(gates[g]):
            if w in last_in_pass:
                assert ppos[last_in_pass[w]] < ppos[g]
            last_in_pass[w] = g
    tb_of_q = {q_: j for j, q_ in enumerate(local)}
    for ph in phases:
        rb, tb = ph["rbits"], ph["tbits"]
        assert rb[0] == 0 and len(rb) == R and sorted(rb + tb) == list(range(k))
        for op in ph["ops"]:
            g = gates[op["gate"]]
            t = tb_of_q[g[1][0]]
            kind = op["kind"]
            if kind in ("ry", "rx", "h", "x", "rz", "cx", "cx_t", "cz", "cz_t"):
                assert rb[op["a"]] == t or (kind in ("cz", "cz_t") and rb[op["a"]] == tb_of_q[g[2][0]])
            if kind == "rz_t":
                assert op["a"] == t and t in tb
            if kind == "cx":
                assert rb[op["b"]] == tb_of_q[g[2][0]]
            if kind == "cx_t":
                assert op["b"] == tb_of_q[g[2][0]] and op["b"] in tb
    # layouts are bijections of the tile
    for m in layouts:
        e = np.arange(1 << k)
        s = e.copy()
        for j in range(k):
            s ^= np.where((e >> j) & 1, m[j], 0)
        assert len(np.unique(s)) == 1 << k
        pair_ok = (s[0::2] ^ 1) == s[1::2]
        assert pair_ok.all(), "neighbouring amplitudes must stay in adjacent words"


@pytest.mark.parametrize("n,kw", [(6, {"k": 4, "contiguous_bits": 2}), (10, {"k": 6}), (14, {"k": 9}),
                                  (16, {"k": 12}), (16, {"k": 10, "rotate_low_bits": True})])
def test_index_maps_are_the_brute_force_permutation(q, n, kw):
    gates = W.ring_ansatz(n, 2)
    p = q.Plan(gates, n, **kw)
    d = p.describe()
    for pi, ps in enumerate(d["passes"][:4]):
        L, NL = ps["L"], ps["nonlocal"]
        # brute force: element index x has bit L[j] = bit j of e, bit NL[j] = bit j of tile
        idx = np.arange(1 << n).reshape((2,) * n)                  # axis a <-> bit n-1-a
        axes = [n - 1 - b for b in reversed(NL)] + [n - 1 - b for b in reversed(L)]
        brute = idx.transpose(axes).reshape(1 << len(NL), 1 << len(L))
        seen = []
        for t in range(1 << len(NL)):
            m = p.tile_index_map(pi, t)
            np.testing.assert_array_equal(m, brute[t])
            seen.append(m)
        assert np.array_equal(np.sort(np.concatenate(seen)), np.arange(1 << n))


@pytest.mark.parametrize("n,layers,kw", [(10, 20, {}), (8, 40, {"contiguous_bits": 2}), (11, 12, {"dtype": "c128"})])
def test_deep_narrow_circuits_rescale_and_split(q, n, layers, kw):
    # a deep circuit on few qubits: passes hold at most MAX_SCALED_PER_PASS unnormalised ops, with a
    # rescale op after every RESCALE_EVERY of them (checked in check_phases)
    gates = W.ring_ansatz(n, layers) + [W.gate(W.H, (i % n,)) for i in range(50)]
    d = q.Plan(gates, n, **kw).describe()
    n_scaled = sum(1 for g in gates if g[0] in (W.RX, W.RY, W.RZ, W.H))
    assert len(d["passes"]) >= -(-n_scaled // MAX_SCALED_PER_PASS)
    n_rescale = 0
    for ps in d["passes"]:
        for key in ("phases", "bwd_phases"):
            check_rescale(gates, ps, ps[key])
        n_rescale += sum(op["kind"] == "scale" for ph in ps["phases"] for op in ph["ops"])
    assert n_rescale >= 1


def test_per_gate_schedule(q):
    gates = W.ring_ansatz(4, 2)
    d = q.Plan(gates, 4, mode="per_gate").describe()
    assert [ps["gates"] for ps in d["passes"]] == [[i] for i in range(len(gates))]


def test_empty_circuit_and_single_qubit(q):
    d = q.Plan([], 3).describe()
    assert len(d["passes"]) == 1 and d["passes"][0]["gates"] == []
    one = [W.gate(W.RX, (0,), param=0), W.gate(W.H, (0,))]
    d1 = q.Plan(one, 1, product_prefix=False).describe()
    assert d1["k"] == 1 and [ps["gates"] for ps in d1["passes"]] == [[0, 1]]
    # with the product prefix both gates become the qubit's prefix state and the one pass has no ops
    d2 = q.Plan(one, 1).describe()
    assert d2["prefix"] == [[0, 1]] and [ps["gates"] for ps in d2["passes"]] == [[]]


@pytest.mark.parametrize("n,kw", [(20, {}), (16, {"dtype": "c128"}), (14, {"k": 10}), (13, {"k": 12}),
                                  (20, {"rotate_low_bits": True}), (18, {"k": 10, "rotate_low_bits": True})])
def test_edge_phases_keep_the_contiguous_run_in_threads(q, n, kw):
    # first and last register phase move data straight between registers and global memory: the tile
    # bits at physical bits 1..3 (the low bits of a contiguous run) must lead the thread bits there so
    # a warp's accesses coalesce
    d = q.Plan(W.ring_ansatz(n, 3), n, **kw).describe()
    for ps in d["passes"]:
        for key, R in (("phases", d["R"]), ("bwd_phases", d["Rb"])):
            if d["k"] - R < 3:
                continue
            # phase 0 moves data in the layout the pass reads, the last phase in the one it writes
            for ph, L in ((ps[key][0], ps["L"]), (ps[key][-1], ps["Lo"])):
                run = [L.index(b) for b in (1, 2, 3)]
                assert not (set(run) & set(ph["rbits"])), (key, ph["rbits"])
                assert ph["tbits"][:3] == run


def test_rotating_low_bits_cut_the_passes():
    # the 20-qubit ring workload at k = 12: the c = 4 coalescing bits are handed between passes
    # instead of holding qubits 16..19 in every tile (24 passes with them fixed)
    import paper_2404_09213_gb300 as qq
    wl = W.config(3)
    assert qq.Plan(wl.gates, wl.n, k=12, rotate_low_bits=True).info()["n_passes"] <= 20
    assert qq.Plan(wl.gates, wl.n, k=11, rotate_low_bits=True).info()["n_passes"] <= 25
    assert qq.Plan(wl.gates, wl.n, k=12, product_prefix=False).info()["n_passes"] == 24
    # the product prefix takes the encoding and the first layer out of the passes: one pass fewer
    assert qq.Plan(wl.gates, wl.n, k=12).info()["n_passes"] == 23


def test_product_prefix_collects_single_qubit_gates_before_first_entangler():
    import paper_2404_09213_gb300 as q
    RX, RY, RZ, H, X, CX, CZ = range(7)
    g = W.gate
    gates = [g(RX, (0,), param=W.input_param(0)), g(RY, (0,), param=0), g(H, (2,)), g(CX, (1,), (0,)),
             g(RZ, (1,), param=1), g(RY, (0,), param=2), g(X, (2,)), g(RZ, (3,), param=3), g(CZ, (3,), (2,)),
             g(RY, (3,), param=4)]
    d = q.Plan(gates, 4, k=3, contiguous_bits=1).describe()
    # qubit 0: RX, RY before CX(0 -> 1); qubit 1: nothing before the CX; qubit 2: H, X before the CZ;
    # qubit 3: RZ before the CZ; the rest stay in the passes
    assert d["prefix"] == [[0, 1], [], [2, 6], [7]]
    in_passes = sorted(i for ps in d["passes"] for i in ps["gates"])
    assert in_passes == [3, 4, 5, 8, 9]
    off = q.Plan(gates, 4, k=3, contiguous_bits=1, product_prefix=False).describe()
    assert off["prefix"] == [] and sorted(i for ps in off["passes"] for i in ps["gates"]) == list(range(10))
    with pytest.raises(q.QsimError):
        q.Plan(gates, 4, mode="per_gate", product_prefix=True)
