"""Multi-process host logic of bench.py (replicas, one process per GPU): two gloo ranks on the CPU.

The fused path has no exchange step between samples or circuits, so N GPUs run N independent
replicas; what needs checking is the launch plumbing: rank/world from the torchrun environment,
the max-over-ranks timing, the barrier, the whole-job aggregate, and that only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["QSIM_ROOT"])
import bench
import torch
import torch.distributed as dist
world, rank, local = bench.dist_init(2)
ms = bench.max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))
bench.barrier(world)
print(json.dumps({"rank": rank, "world": world, "local": local, "backend": dist.get_backend(),
                  "ms_max": ms, "value": bench.replica_value(world, 64, 10, ms)}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(argv, n=2, timeout=300):
    port = free_port()
    procs = []
    for r in range(n):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(n), RANK=str(r),
                   LOCAL_RANK=str(r), QSIM_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable] + argv, env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            outs.append((p.returncode, out, err))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


def test_two_gloo_ranks_max_over_ranks_and_aggregate():
    outs = run_ranks(["-c", WORKER])
    recs = []
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
        recs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(r["rank"] for r in recs) == [0, 1]
    for r in recs:
        assert r["world"] == 2 and r["local"] == r["rank"] and r["backend"] == "gloo"
        assert r["ms_max"] == 20.0                     # the slower rank's time
        assert r["value"] == 2 * 64 * 10 / 0.020       # both replicas' samples over that time


def test_reference_arm_prints_once_under_two_ranks():
    outs = run_ranks(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    (rc0, out0, err0), (rc1, out1, err1) = outs
    assert rc0 == 0, err0[-2000:]
    assert rc1 == 0, err1[-2000:]
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert out1.strip() == ""
