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


def test_pass_roofline_on_the_bench_plan():
    # the bench's roofline object, from the real 20-qubit plan description and synthetic event times
    import json
    import numpy as np
    import workloads as W
    from paper_2404_09213_gb300 import build
    build.build()
    import paper_2404_09213_gb300 as q
    wl = W.config(3)
    plan = q.Plan(wl.gates, wl.n, k=12, checkpoint_passes=1)
    desc = plan.describe()
    P = len(desc["passes"])
    fwd_ms = np.full(P, 0.2 * 3)            # 3 recorded calls of 0.2 ms per pass
    bwd_ms = np.full(P, 0.6 * 3)
    r = bench.pass_roofline(desc, wl.batch, wl, 1, "fused", fwd_ms, bwd_ms, 3, 3, "// not the measured program",
                            6758.5, "measured")
    json.dumps(r)
    amps = wl.batch * (1 << wl.n)
    bb = bench.algorithmic_bytes(desc, wl.batch, wl.n, "bwd", 1)
    assert r["kernel"] == "bwd_pass_kernel" and r["launches_timed"] == 3 * P and r["traffic"] is None
    assert abs(r["avg_launch_ms"] - 0.6) < 1e-12
    assert abs(r["achieved"] - sum(bb) / P / 0.6e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6758.5) < 1e-12
    assert r["bytes_per_gate"]["per_gate_path_fwd"] == 16 * amps
    assert r["per_pass"]["gates"] == [len(ps["gates"]) for ps in desc["passes"]]
    # every gate runs in a pass or was merged into a qubit's prefix state (the first pass starts from it)
    assert sum(r["per_pass"]["gates"]) + sum(len(x) for x in desc["prefix"]) == len(wl.gates)


def test_alu_roofline():
    # 3.93 GFLOP per step in 0.2 ms of pass-kernel time (two recorded calls of one pass) at an 80 TFLOP/s peak
    r = bench.alu_roofline(3.93e9, [0.4], 2, 0.25, 80.0, "derived")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["launches_timed"] == 2
    assert abs(r["achieved"] - 3.93e9 / 0.2e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 80.0) < 1e-12
    assert abs(r["pass_kernel_share_of_step"] - 0.8) < 1e-12
