"""Host arithmetic of bench.py: algorithmic bytes per pass, the per-pass table, the traffic record."""
import bench


def fake_desc(gates_per_pass):
    return {"passes": [{"gates": list(range(g))} for g in gates_per_pass]}


def test_algorithmic_bytes_forward_and_backward():
    d = fake_desc([5, 7, 3, 4])
    amps = 2 * (1 << 3)
    # forward: the first pass starts from |0> and only writes
    assert bench.algorithmic_bytes(d, 2, 3, "fwd") == [8 * amps, 16 * amps, 16 * amps, 16 * amps]
    # backward without checkpoints: pass P-1 reads psi only and writes psi, lambda; pass 0 writes nothing
    assert bench.algorithmic_bytes(d, 2, 3, "bwd") == [16 * amps, 32 * amps, 32 * amps, 24 * amps]
    # a checkpoint every pass: psi is never stored back
    assert bench.algorithmic_bytes(d, 2, 3, "bwd", 1) == [16 * amps, 24 * amps, 24 * amps, 16 * amps]
    # every second pass: the passes whose predecessor restarts from a checkpoint skip the psi store
    assert bench.algorithmic_bytes(d, 2, 3, "bwd", 2) == [16 * amps, 32 * amps, 24 * amps, 24 * amps]


def test_per_pass_table():
    d = fake_desc([4, 0, 10])
    t = bench.per_pass_table(d, [4000, 8000, 10000], [6000, 9000, 3000], [2e-6 * 2, 4e-6 * 2, 0.0],
                             [3e-6 * 2, 0.0, 1e-6 * 2], 2, 2)
    assert t["gates"] == [4, 0, 10]
    assert t["bytes_per_gate_fwd"] == [1000, 8000, 1000]
    # 4000 B in 2e-6 ms = 2e-9 s -> 2000 GB/s
    assert t["fwd_gbs"] == [2000.0, 2000.0, None]
    assert t["bwd_gbs"] == [2000.0, None, 3000.0]


def test_traffic_record_needs_the_measured_kernel_program():
    assert bench.traffic_record("bwd_pass_kernel", "// some other program") is None
    assert bench.traffic_record("no_such_kernel", "") is None
