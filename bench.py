#!/usr/bin/env python
"""Throughput benchmark: forward + adjoint backward of a 20-qubit, 64-sample batch.

Workload (``C3``): RX angle encoding of 20 inputs, then 10 layers of (RY, RZ on every qubit) +
CNOT ring; complex64 state (512 MiB per batch, larger than L2), float64 <Z_i> and gradients.
One step = qsim_forward (angle -> coefficients, fused passes, <Z> reduction) + qsim_backward
(adjoint passes, gradient reductions) on device-resident inputs. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode fused|per_gate]

For N > 1 launch under torchrun: every rank runs its own replica (the method has no exchange
step on one circuit batch), rank 0 prints the line, ``value`` sums over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint-bwd samples/s"
UNIT = "samples/s"
WORKLOAD = "C3: 20 qubits, batch 64, complex64, RX encoding + 10 x (RY,RZ per qubit + CNOT ring), fwd+bwd"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fused", choices=["fused", "per_gate"])
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--batch", type=int, default=64, help="samples (64 = the workload; smaller for ncu captures)")
    ap.add_argument("--workload", default="c3", choices=["c2", "c3", "c4", "c5", "sel", "landscape"],
                    help="c3 (default): 20 qubits x 64, fwd+bwd; c2: 12 qubits x 1024 forward; "
                         "c4: 256 circuits (8..22 qubits) x 4 in one persistent launch, fwd+bwd; "
                         "c5: 30 qubits x 1, fwd + checkpointed bwd; sel: 20 qubits x 64, Strongly Entangling "
                         "Layers with data re-uploading, fwd+bwd; landscape: every parameter of a 5-qubit SEL "
                         "circuit swept over 256 values (qsim_landscape)")
    ap.add_argument("--contiguous-bits", type=int, default=0)
    ap.add_argument("--checkpoint-passes", type=int, default=1,
                    help="store the state every this many forward passes (1: every pass, so backward passes "
                         "read stored states instead of writing uncomputed ones; 0: none)")
    ap.add_argument("--no-pauli-frame", action="store_true",
                    help="fused passes pick each rotation's tangent or cotangent form per sample at run time "
                         "(default: the tangent form only, cotangent Paulis carried in a per-sample frame)")
    ap.add_argument("--scalar-bwd", action="store_true",
                    help="backward pass kernels update psi and lambda with scalar FMAs (default: packed FP32x2 pairs)")
    ap.add_argument("--no-product-prefix", action="store_true",
                    help="run every gate inside the fused passes (default: single-qubit gates before a qubit's first "
                         "two-qubit gate are merged into its prefix state and the first pass starts from the product)")
    ap.add_argument("--split-diagonal", action="store_true",
                    help="apply runs of diagonal ops one op at a time (default: one factor per amplitude per run)")
    ap.add_argument("--max-regs", type=int, default=0,
                    help="cap the pass kernels' registers per thread (0: the compiler's choice)")
    ap.add_argument("--bwd-reg-bits", type=int, default=0, help="amplitudes per thread in backward phases = 2^bits (0: default)")
    ap.add_argument("--fwd-reg-bits", type=int, default=0, help="amplitudes per thread in forward phases = 2^bits (0: default)")
    ap.add_argument("--large-qubits", type=int, default=0,
                    help="c4: circuits of at least this many qubits run as their own single-circuit plan "
                         "(0: the library default, -1: every circuit in the persistent queue)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-gate", action="store_true", help="skip timing the per-gate path next to the fused one")
    ap.add_argument("--per-gate-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--json-out", default="")
    ap.add_argument("--oracle-table", action="store_true",
                    help="with --impl reference: time the FP64 oracles on the host cores over every configuration "
                         "(Oracle-K: C1, C2 on samples 0..31, the 12-qubit C3 / C5 ansatze; Oracle-S: C3) and print "
                         "one JSON line")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed plumbing
def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, samples_per_rank, steps, ms_max):
    """Whole-job samples/s of `world` replicas, each processing `samples_per_rank` samples per step,
    timed by the slowest rank (ms_max over `steps` steps)."""
    return world * samples_per_rank * steps / (ms_max / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join("/tmp", f"qsim_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle (bounded sample)
def _oracle_job(args):
    """One sample's forward + adjoint backward through a gate list (FP64 oracle); seconds."""
    gates, n, params, x_row, g_row = args
    import oracle
    t0 = time.perf_counter()
    oracle.grad_adjoint(gates, n, params, x_row[None, :], g_row[None, :])
    return time.perf_counter() - t0


def _oracle_pool(cores):
    import multiprocessing as mp
    # spawn: the parent has used CUDA, and a forked child of such a process can hang
    pool = mp.get_context("spawn").Pool(cores)
    pool.map(_oracle_job, [([], 1, np.zeros(0), np.zeros(1), np.zeros(1))] * cores)   # import oracle in every worker
    return pool


def oracle_bounded(wl, pool, cores, per_core_s=1.5, calib=None):
    """The FP64 oracle's forward + adjoint backward (oracle.grad_adjoint), one sample per host core in
    parallel, over a window of the circuit sized to ~per_core_s seconds per core; extrapolated to the
    whole circuit (its cost is a sum over gates). Returns (samples/s, wall seconds, description)."""
    G = len(wl.gates)
    if calib is None:
        calib = _oracle_job((wl.gates[:20], wl.n, wl.params, wl.inputs[0], wl.grad_out[0])) / 20
    g_t = max(4, min(G, int(per_core_s / max(calib, 1e-6))))
    a = max(0, min(G - g_t, G // 2 - g_t // 2))   # a window from the middle: every gate kind of the circuit
    jobs = [(wl.gates[a:a + g_t], wl.n, wl.params, wl.inputs[b % wl.batch], wl.grad_out[b % wl.batch])
            for b in range(cores)]
    t0 = time.perf_counter()
    pool.map(_oracle_job, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    rate = cores / (wall * G / g_t)
    desc = (f"FP64 oracle (numpy, strided gates; forward + adjoint backward, oracle.grad_adjoint): {cores} samples in "
            f"parallel processes, one per host core, each through gates {a}..{a + g_t - 1} of {G} (from |0...0>) in {wall:.2f} s wall; "
            f"extrapolated x{G / g_t:.2f} to the whole circuit")
    return rate, wall, desc, {"extrapolated": True, "gates_timed": g_t, "gates_total": G, "samples_timed": cores,
                              "wall_s_timed": wall}, calib


def _oracle_window_job(args):
    """Seconds for one oracle call: method 'kron' / 'strided' forward, or 'adjoint' fwd+bwd, over a gate list."""
    method, gates, n, params, inputs, g = args
    import oracle
    t0 = time.perf_counter()
    if method == "adjoint":
        oracle.grad_adjoint(gates, n, params, inputs, g)
    elif method == "kron":
        oracle.simulate_kron(gates, n, params, inputs)
    else:
        oracle.simulate_strided(gates, n, params, inputs)
    return time.perf_counter() - t0


def oracle_table(cores, budget_s=8.0):
    """Samples/s of the FP64 oracles per configuration, each from a timed window of the circuit scaled to
    the whole circuit (forward: x G / g; parameter-shift backward: 2 forwards per rotation), the windows
    of one row run as parallel processes (one per core, each on its own samples)."""
    import workloads as W
    pool = _oracle_pool(cores)
    rows = []

    def window(wl, method, samples_per_job, jobs):
        G = len(wl.gates)
        one = _oracle_window_job((method, wl.gates[:4], wl.n, wl.params, wl.inputs[:samples_per_job],
                                  wl.grad_out[:samples_per_job])) / 4
        g_t = max(4, min(G, int(budget_s / max(one, 1e-6))))
        a = max(0, min(G - g_t, G // 2 - g_t // 2))
        args = [(method, wl.gates[a:a + g_t], wl.n, wl.params,
                 wl.inputs[(j * samples_per_job) % wl.batch:][:samples_per_job],
                 wl.grad_out[(j * samples_per_job) % wl.batch:][:samples_per_job]) for j in range(jobs)]
        t0 = time.perf_counter()
        pool.map(_oracle_window_job, args, chunksize=1)
        wall = time.perf_counter() - t0
        return wall * G / g_t, g_t, G, wall

    def add(name, wl, method, spj, jobs, shift_factor, what):
        t_full, g_t, G, wall = window(wl, method, spj, jobs)
        samples = spj * jobs
        rate = samples / (t_full * shift_factor)
        rows.append({"config": name, "oracle": what, "samples_per_s": rate, "samples_timed": samples,
                     "gates_timed": g_t, "gates_total": G, "wall_s_timed": wall,
                     "extrapolated": g_t < G or shift_factor != 1})

    c1 = W.config(1)
    n_rot1 = sum(1 for gt in c1.gates if gt[0] <= 2)
    add("C1 4q B8 c128", c1, "kron", c1.batch, 1, 1 + 2 * n_rot1, "Oracle-K forward + parameter-shift backward")
    c2 = W.config(2)
    add("C2 12q, samples 0..31", c2, "kron", 32 // cores if cores <= 32 else 1, min(cores, 32), 1, "Oracle-K forward")
    for c in (3, 5):
        wl = W.config(c, n=12, batch=max(2, cores))
        n_rot = sum(1 for gt in wl.gates if gt[0] <= 2)
        add(f"C{c} ansatz at 12 qubits", wl, "kron", 1, cores, 1 + 2 * n_rot, "Oracle-K forward + parameter-shift backward")
        add(f"C{c} ansatz at 12 qubits", wl, "adjoint", 1, cores, 1, "Oracle-S forward + adjoint backward")
    c3 = W.config(3)
    add("C3 20q, samples 0..15", c3, "strided", 1, min(cores, 16), 1, "Oracle-S forward")
    pool.close()
    return rows


# ------------------------------------------------------------------ our arm
def algorithmic_bytes(plan_desc, B, n, direction, checkpoint_passes=0):
    """Bytes each fused pass must move (complex64, 8 B per amplitude and state read or written).

    Forward: read + write (the first pass starts from |0> and only writes). Backward pass q: reads psi
    and lambda (the last pass, which runs first, forms lambda from psi), writes lambda (not pass 0) and
    psi unless q == 0 or the pass before it restarts from a stored checkpoint (q a multiple of the
    checkpoint spacing)."""
    P = len(plan_desc["passes"])
    amps = B * (1 << n)
    if direction == "fwd":
        return [amps * (8 if q == 0 else 16) for q in range(P)]
    m = checkpoint_passes
    out = []
    for q in range(P):
        rd = 8 + (8 if q < P - 1 else 0)
        wr = (8 if q > 0 else 0) + (8 if q > 0 and not (m > 0 and q % m == 0) else 0)
        out.append(amps * (rd + wr))
    return out


def per_pass_table(desc, fwd_bytes, bwd_bytes, fwd_ms, bwd_ms, n_fwd, n_bwd):
    """Per fused pass: gates, HBM bytes per gate (forward), and achieved GB/s in each direction from the
    pass's own event-timed launches (ms summed over n_fwd / n_bwd recorded calls)."""
    gates = [len(ps["gates"]) for ps in desc["passes"]]
    f_ms = [float(t) / max(n_fwd, 1) for t in fwd_ms]
    b_ms = [float(t) / max(n_bwd, 1) for t in bwd_ms]
    return {"gates": gates,
            "bytes_per_gate_fwd": [round(fb / max(g, 1)) for fb, g in zip(fwd_bytes, gates)],
            "fwd_gbs": [round(fb / (t / 1e3) / 1e9, 1) if t > 0 else None for fb, t in zip(fwd_bytes, f_ms)],
            "bwd_gbs": [round(bb / (t / 1e3) / 1e9, 1) if t > 0 else None for bb, t in zip(bwd_bytes, b_ms)]}


def pass_roofline(desc, B, wl, ckpt, mode, fwd_ms, bwd_ms, nf, nb, kernel_source, peak, peak_kind):
    """Roofline object of the dominant pass kernel (backward in fused mode): algorithmic bytes per launch
    over its average event-timed launch, against the measured HBM peak; plus bytes per gate and the
    per-pass table. fwd_ms / bwd_ms: per-pass event times summed over nf / nb recorded calls."""
    fb = algorithmic_bytes(desc, B, wl.n, "fwd")
    bb = algorithmic_bytes(desc, B, wl.n, "bwd", ckpt)
    kern = "bwd_pass_kernel" if mode == "fused" else "pg_bwd_kernel"
    if fwd_ms.sum() > bwd_ms.sum():
        kern = "fwd_pass_kernel" if mode == "fused" else "pg_gate_kernel"
        tot_b, tot_ms, n_l = sum(fb) * nf, float(fwd_ms.sum()), len(fb) * nf
    else:
        tot_b, tot_ms, n_l = sum(bb) * nb, float(bwd_ms.sum()), len(bb) * nb
    achieved = (tot_b / n_l) / ((tot_ms / n_l) / 1e3) / 1e9 if tot_ms > 0 else None
    return {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic_record(kern, kernel_source),
            "kernel_source_sha256": hashlib.sha256(kernel_source.encode()).hexdigest(),
            "algorithmic_bytes_per_launch": tot_b / n_l if n_l else None,
            "avg_launch_ms": tot_ms / n_l if n_l else None, "launches_timed": n_l,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
            "fwd_ms_per_step": float(fwd_ms.sum()) / max(nf, 1), "bwd_ms_per_step": float(bwd_ms.sum()) / max(nb, 1),
            "passes": len(desc["passes"]),
            # HBM bytes per gate: fused passes amortise one round trip over all of a pass's gates
            "bytes_per_gate": {"fwd": sum(fb) / len(wl.gates), "bwd": sum(bb) / len(wl.gates),
                               "per_gate_path_fwd": 16 * B * (1 << wl.n),
                               "per_gate_path_bwd": 32 * B * (1 << wl.n)},
            "per_pass": per_pass_table(desc, fb, bb, fwd_ms, bwd_ms, nf, nb) if mode == "fused" else None}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def alu_roofline(flops_per_step, fwd_ms, n_fwd, step_ms, peak_tflops, peak_source):
    """Roofline on the FP32 ALUs of the forward pass kernels: algorithmic flops per step over their
    event time per step (fwd_ms: per-pass times summed over n_fwd recorded calls)."""
    P = len(fwd_ms)
    kern_ms = float(sum(fwd_ms)) / max(n_fwd, 1)
    ach = flops_per_step / (kern_ms / 1e3) / 1e12 if kern_ms > 0 else None
    return {"bound": "alu", "kernel": "fwd_pass_kernel", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": ach / peak_tflops if ach else None, "traffic": None,
            "algorithmic_flops_per_launch": flops_per_step / P, "avg_launch_ms": kern_ms / P,
            "launches_timed": n_fwd * P, "peak_source": peak_source,
            "pass_kernel_share_of_step": kern_ms / step_ms if step_ms > 0 else None}


def fp32_peak_tflops(dev_index):
    """FP32 peak derived from unit counts and clocks: SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
    (the maximum SM clock of this GPU model)."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    return sms * 128 * 2 * 2.070e9 / 1e12, f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz"


def traffic_record(kernel, kernel_source):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if the plan's generated kernel
    program (every pass kernel, as compiled) is the one the counters were taken on."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    if rec.get("kernel_source_sha256") != hashlib.sha256(kernel_source.encode()).hexdigest():
        return None
    return rec.get("dram_bytes_per_launch_full")


def c3_config(wl, world):
    """The workload as both arms name it (implementation choices are reported under "plan")."""
    return {"workload": WORKLOAD, "n_qubits": wl.n, "batch": wl.batch, "gates": len(wl.gates),
            "params": wl.n_params, "inputs_per_sample": wl.n_inputs,
            "l2": "inputs larger than L2: 512 MiB state per step (L2 129 MB), no flush needed",
            "parallelism": f"replicas x{world}"}


def run_ours(args, world, rank, local):
    import torch
    import workloads as W
    from paper_2404_09213_gb300 import build as qbuild
    qbuild.build()
    import paper_2404_09213_gb300 as q

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.config(3, batch=args.batch)
    k, autotune = args.k, None
    if args.mode == "fused" and k == 0:   # tile size from the library's autotuner (untimed setup)
        k, ms = q.autotune(wl.gates, wl.n, wl.batch, reps=2, contiguous_bits=args.contiguous_bits,
                           checkpoint_passes=args.checkpoint_passes, pauli_frame=int((not args.no_pauli_frame)),
                           scalar_bwd=int(args.scalar_bwd), product_prefix=int(not args.no_product_prefix),
                           bwd_reg_bits=args.bwd_reg_bits, fwd_reg_bits=args.fwd_reg_bits,
                           split_diagonal=int(args.split_diagonal), max_regs=args.max_regs)
        autotune = {"k_candidates": [11, 12, 13], "ms_per_fwd_bwd": ms[:3], "chosen_k": k}
    ckpt = args.checkpoint_passes if args.mode == "fused" else 0
    plan = q.Plan(wl.gates, wl.n, dtype="c64", mode=args.mode, k=k, contiguous_bits=args.contiguous_bits,
                  checkpoint_passes=ckpt, pauli_frame=(not args.no_pauli_frame) and args.mode == "fused",
                  scalar_bwd=args.scalar_bwd, product_prefix=args.mode == "fused" and not args.no_product_prefix,
                  bwd_reg_bits=args.bwd_reg_bits, fwd_reg_bits=args.fwd_reg_bits, split_diagonal=args.split_diagonal,
                  max_regs=args.max_regs)
    desc = plan.describe()
    p = torch.tensor(wl.params, dtype=torch.float32, device=dev)
    x = torch.tensor(wl.inputs, dtype=torch.float32, device=dev)
    g = torch.tensor(wl.grad_out, dtype=torch.float64, device=dev)
    B = wl.batch
    states = torch.empty((B, 1 << wl.n), dtype=torch.complex64, device=dev)
    z = torch.empty((B, wl.n), dtype=torch.float64, device=dev)
    dp = torch.empty((wl.n_params,), dtype=torch.float64, device=dev)
    di = torch.empty((B, wl.n_inputs), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.forward(p, x, states=states, z=z, stream=stream)
        plan.backward(g, dparams=dp, dinputs=di, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    plan.set_profiling(args.steps)
    clk = ClockSampler(local)
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = q.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = q.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    fwd_ms, bwd_ms, nf, nb = plan.read_profile()
    plan.set_profiling(0)
    ms_max = max_over_ranks(ms, world, dev)
    value = replica_value(world, B, args.steps, ms_max)

    # roofline of the dominant kernel (fused backward pass kernel in fused mode)
    peak, peak_kind = load_peaks()
    roofline = pass_roofline(desc, B, wl, ckpt, args.mode, fwd_ms, bwd_ms, nf, nb, plan.kernel_source(), peak, peak_kind)

    # end to end: host inputs -> device, forward + backward, results -> host, every step
    e2e = None
    if not args.no_e2e:
        hp = torch.tensor(wl.params, dtype=torch.float32).pin_memory()
        hx = torch.tensor(wl.inputs, dtype=torch.float32).pin_memory()
        hg = torch.tensor(wl.grad_out, dtype=torch.float64).pin_memory()
        hz = torch.empty((B, wl.n), dtype=torch.float64).pin_memory()
        hdp = torch.empty((wl.n_params,), dtype=torch.float64).pin_memory()
        hdi = torch.empty((B, wl.n_inputs), dtype=torch.float64).pin_memory()

        def e2e_step():
            p.copy_(hp, non_blocking=True)
            x.copy_(hx, non_blocking=True)
            g.copy_(hg, non_blocking=True)
            step()
            hz.copy_(z, non_blocking=True)
            hdp.copy_(dp, non_blocking=True)
            hdi.copy_(di, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        barrier(world)
        sec = max_over_ranks(t1 - t0, world, dev)
        h2d = hp.numel() * 4 + hx.numel() * 4 + hg.numel() * 8
        d2h = hz.numel() * 8 + hdp.numel() * 8 + hdi.numel() * 8
        e2e = {"value": replica_value(world, B, args.steps, sec * 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # the plain one-kernel-per-gate path on the same GPU, same workload and precision, timed in this
    # process (the denominator of the fused path's speed-up)
    per_gate = None
    if args.mode == "fused" and not args.no_per_gate:
        pg = q.Plan(wl.gates, wl.n, dtype="c64", mode="per_gate")

        def pg_step():
            pg.forward(p, x, states=states, z=z, stream=stream)
            pg.backward(g, dparams=dp, dinputs=di, stream=stream)
        for _ in range(3):
            pg_step()
        torch.cuda.synchronize()
        barrier(world)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.per_gate_steps):
            pg_step()
        f1.record(stream)
        torch.cuda.synchronize()
        pg_ms = max_over_ranks(f0.elapsed_time(f1), world, dev) / args.per_gate_steps
        pg_value = replica_value(world, B, 1, pg_ms)
        per_gate = {"value": value / pg_value, "unit": "x (fused samples/s over per-gate samples/s)",
                    "per_gate_samples_per_s": pg_value, "per_gate_ms_per_step": pg_ms,
                    "steps": args.per_gate_steps, "warmup": 3,
                    "path": "one kernel per gate over the whole batch, same precision and reductions"}
        del pg

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded splitmix64 angles and loss weights)",
           "config": c3_config(wl, world),
           "plan": {"mode": args.mode, "k": desc["k"], "autotune": autotune,
                    "precision": "complex64 state, FP32 arithmetic; <Z> and gradient sums FP32 within a tile, "
                                 "FP64 across tiles and samples",
                    "checkpoint_passes": ckpt, "checkpoints": plan.info()["n_checkpoints"],
                    "pauli_frame": bool((not args.no_pauli_frame) and args.mode == "fused"),
                    "packed_bwd": bool((not args.no_pauli_frame) and args.mode == "fused" and not args.scalar_bwd),
                    "product_prefix": bool(args.mode == "fused" and not args.no_product_prefix),
                    "merged_diagonal_runs": bool((not args.no_pauli_frame) and args.mode == "fused" and not args.split_diagonal),
                    "prefix_gates": sum(len(x) for x in desc.get("prefix", [])),
                    "reg_bits": {"fwd": desc.get("R"), "bwd": desc.get("Rb")}, "max_regs": args.max_regs,
                    "workspace_bytes": plan.info()["workspace_bytes"], "contiguous_bits": desc["c"]},
           "roofline": roofline, "vs_per_gate": per_gate, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    return out, wl


def run_other(args, world, rank, local):
    """Secondary workloads (one JSON line each): C2 forward, C4 multi-circuit, C5 30 qubits."""
    import torch
    import workloads as W
    from paper_2404_09213_gb300 import build as qbuild
    qbuild.build()
    import paper_2404_09213_gb300 as q
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = load_peaks()
    if args.workload == "c4":
        wls = W.multi_circuit_config()
        B = 4
        circuits = [(w.gates, w.n) for w in wls]
        ks = q.multi_autotune(circuits, B, reps=2)   # per qubit count (untimed setup)
        mp = q.MultiPlan(circuits, graph=True, ks=ks, large_qubits=args.large_qubits)
        p = torch.tensor(np.concatenate([w.params for w in wls]), dtype=torch.float32, device=dev)
        x = torch.tensor(np.concatenate([w.inputs.ravel() for w in wls]), dtype=torch.float32, device=dev)
        g = torch.tensor(np.concatenate([w.grad_out.ravel() for w in wls]), dtype=torch.float64, device=dev)
        off = mp.offsets(B)
        states = torch.empty(int(off["states"][-1]), dtype=torch.complex64, device=dev)
        z = torch.empty(int(off["z"][-1]), dtype=torch.float64, device=dev)
        dp = torch.zeros(int(off["params"][-1]), dtype=torch.float64, device=dev)
        di = torch.zeros(int(off["inputs"][-1]), dtype=torch.float64, device=dev)

        def step():
            mp.forward(p, x, B, states=states, z=z, stream=stream)
            mp.backward(g, dparams=dp, dinputs=di, stream=stream)
        samples = B * len(wls)
        # algorithmic bytes of every pass (complex64): forward 16 B/amp (8 for the |0> start),
        # backward 32 B/amp (24 for the first, 16 for the last)
        tot = 0
        for w, kc in zip(wls, ks):
            P = q.Plan(w.gates, w.n, k=kc).info()["n_passes"]
            amps = B * (1 << w.n)
            tot += amps * (8 + 16 * (P - 1))
            tot += amps * (8 if P == 1 else 24 + 16 + 32 * (P - 2))
        name = "C4: 256 circuits, 8..22 qubits (log-uniform), depth 4..16, HEA (RY,RZ + CZ ladder), batch 4, c64, fwd+bwd"
        extra = {"circuits": len(wls), "batch_per_circuit": B, "graph": True, "large_qubits": args.large_qubits,
                 "k_by_qubits": {str(w.n): kc for w, kc in sorted(zip(wls, ks), key=lambda t: t[0].n)}}
    elif args.workload == "c5":
        wl = W.config(5)
        B = 1
        plan = q.Plan(wl.gates, wl.n, checkpoint_passes=8)
        p = torch.tensor(wl.params, dtype=torch.float32, device=dev)
        x = torch.tensor(wl.inputs, dtype=torch.float32, device=dev)
        g = torch.tensor(wl.grad_out, dtype=torch.float64, device=dev)

        def step():
            plan.forward(p, x, stream=stream)
            plan.backward(g, stream=stream)
        samples = B
        P = plan.info()["n_passes"]
        desc = plan.describe()
        tot = sum(algorithmic_bytes(desc, B, wl.n, "fwd")) + sum(algorithmic_bytes(desc, B, wl.n, "bwd", 8))
        name = "C5: 30 qubits, batch 1, c64, RX encoding + 8 x (RY,RZ + CNOT ring), fwd + checkpointed bwd"
        extra = {"passes": P, "checkpoint_passes": 8}
    elif args.workload == "sel":
        wl = W.sel_workload("SEL", 20, 64, 5, "c64", seed=W.SEED_BASE + 6, reupload=True)
        B = wl.batch
        k, _ = q.autotune(wl.gates, wl.n, B, reps=2, checkpoint_passes=1)
        plan = q.Plan(wl.gates, wl.n, k=k, checkpoint_passes=1)
        p = torch.tensor(wl.params, dtype=torch.float32, device=dev)
        x = torch.tensor(wl.inputs, dtype=torch.float32, device=dev)
        g = torch.tensor(wl.grad_out, dtype=torch.float64, device=dev)
        states = torch.empty((B, 1 << wl.n), dtype=torch.complex64, device=dev)
        z = torch.empty((B, wl.n), dtype=torch.float64, device=dev)

        def step():
            plan.forward(p, x, states=states, z=z, stream=stream)
            plan.backward(g, stream=stream)
        samples = B
        desc = plan.describe()
        tot = sum(algorithmic_bytes(desc, B, wl.n, "fwd")) + sum(algorithmic_bytes(desc, B, wl.n, "bwd", 1))
        name = ("SEL: 20 qubits, batch 64, c64, 5 Strongly Entangling Layers (Rot + range-r CNOTs) with data "
                "re-uploading before every layer, fwd+bwd")
        extra = {"passes": len(desc["passes"]), "k": k, "gates": len(wl.gates), "params": wl.n_params,
                 "checkpoint_passes": 1}
    elif args.workload == "landscape":
        n, layers, V = 5, 5, 256
        gates = W.sel_ansatz(n, layers, encode=False)
        P = W.count_params(gates)
        rng = W.SplitMix64(W.SEED_BASE + 7)
        base = torch.tensor(rng.uniforms(P) * 2 * math.pi - math.pi, dtype=torch.float32, device=dev)
        values = torch.linspace(-math.pi, math.pi, V, device=dev)
        weights = torch.ones(n, dtype=torch.float64, device=dev)

        def step():
            q.landscape(gates, n, base, values, weights, weight_remap=True, stream=stream)
        samples = P * V
        B = P * V
        tot = B * (1 << n) * (8 + 24)   # one pass each way (whole 5-qubit state in one tile)
        name = (f"gradient landscape: {P} parameters of a 5-qubit, {layers}-layer SEL circuit, each swept over "
                f"{V} values with the others fixed, weight remapping (one qsim_landscape call per step, plan "
                "and kernel loading included)")
        extra = {"params": P, "values": V, "gradient_vectors_per_step": P * V}
    else:
        wl = W.config(2)
        B = wl.batch
        tuned = {}
        if args.mode == "fused":   # one pass: the autotuner picks the register bits (untimed setup)
            _, c2_ms, tuned = q.autotune(wl.gates, wl.n, B, with_backward=False, reps=3, return_opts=True,
                                         pauli_frame=int(not args.no_pauli_frame))
        if not tuned:
            tuned = {"pauli_frame": (not args.no_pauli_frame) and args.mode == "fused"}
        plan = q.Plan(wl.gates, wl.n, mode=args.mode, **tuned)
        p = torch.tensor(wl.params, dtype=torch.float32, device=dev)
        x = torch.tensor(wl.inputs, dtype=torch.float32, device=dev)
        states = torch.empty((B, 1 << wl.n), dtype=torch.complex64, device=dev)
        z = torch.empty((B, wl.n), dtype=torch.float64, device=dev)

        def step():
            plan.forward(p, x, states=states, z=z, stream=stream)
        samples = B
        P = plan.info()["n_passes"]
        tot = B * (1 << wl.n) * (8 + 16 * (P - 1)) if args.mode == "fused" else B * (1 << wl.n) * 16 * len(wl.gates)
        # algorithmic work of the pass kernel: a real 2x2 rotation costs 6 flop per amplitude (CNOTs are
        # permutations), counted over the rotations the pass applies (not those merged into prefix states)
        desc = plan.describe()
        n_rot = sum(1 for ps in desc["passes"] for gi in ps["gates"] if wl.gates[gi][0] in (W.RX, W.RY, W.RZ))
        n_rot_circuit = sum(1 for gt in wl.gates if gt[0] in (W.RX, W.RY, W.RZ))
        c2_flops = B * (1 << wl.n) * 6 * n_rot
        name = f"C2: 12 qubits, batch 1024, c64, RX encoding + 6 x (RY,RZ + CNOT ring), forward only, {args.mode}"
        extra = {"passes": P, "mode": args.mode, "rotations_in_passes": n_rot, "rotations": n_rot_circuit,
                 "autotune": {"candidates": ["2^5 with the frame", "2^4 with the frame", "2^5 without", "2^4 without"], "ms": c2_ms,
                              **tuned} if args.mode == "fused" else None,
                 "prefix_gates": sum(len(x) for x in desc.get("prefix", [])),
                 "l2": "32 MiB state per step stays in L2 and shared memory (ALU-bound, no flush)"}
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if args.workload == "c4":
        extra["queue"] = mp.info()
    c2_profile = args.workload == "c2" and args.mode == "fused"
    if c2_profile:
        plan.set_profiling(args.steps)
    clk = ClockSampler(local)
    time.sleep(0.3)
    launches0 = q.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    launches = q.kernel_launches() - launches0
    gbs = tot * args.steps / (ms / 1e3) / 1e9
    metric = {"c2": "forward samples/s", "landscape": "gradient vectors/s"}.get(args.workload, "fwd+adjoint-bwd samples/s")
    unit = "gradient vectors/s" if args.workload == "landscape" else UNIT
    roofline = {"bound": "hbm", "kernel": "whole step (all pass kernels)", "achieved": gbs, "peak": peak,
                "unit": "GB/s", "frac": gbs / peak, "traffic": None,
                "algorithmic_bytes_per_step": tot, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    if c2_profile:
        # the state never leaves L2 / shared memory: a roofline on the FP32 ALUs for the pass kernel
        fwd_ms, _, nf, _ = plan.read_profile()
        plan.set_profiling(0)
        roofline = alu_roofline(c2_flops, fwd_ms, nf, ms / args.steps, *fp32_peak_tflops(local))
    out = {"metric": metric, "value": samples * args.steps / (ms / 1e3), "unit": unit, "n_gpus": 1,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded splitmix64)",
           "config": dict(workload=name, precision="complex64 state, FP32 arithmetic, FP64 sums across tiles", **extra),
           "roofline": roofline, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out))


def main():
    args = parse()
    world, rank, local = dist_init(args.gpus)
    if args.impl == "reference" and args.oracle_table:
        if rank == 0:
            cores = os.cpu_count() or 1
            print(json.dumps({"oracle_table": oracle_table(cores), "cores": cores}))
        return
    if args.impl == "reference":
        if rank != 0:
            return
        import workloads as W
        wl = W.config(3)
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        pool = _oracle_pool(cores)
        calib = None
        for _ in range(args.warmup):
            _, _, _, _, calib = oracle_bounded(wl, pool, cores, per_core_s=0.2, calib=calib)
        rates, walls = [], []
        for _ in range(args.steps):
            r, wall, sample, ext, calib = oracle_bounded(wl, pool, cores, calib=calib)
            rates.append(r)
            walls.append(wall)
        pool.close()
        dt = time.perf_counter() - t0
        v = statistics.median(rates)
        ext["steps_timed"] = args.steps
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded splitmix64)",
                "config": c3_config(wl, 1),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample, **ext},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "note": "each step runs the bounded sample above (ms_per_step is its wall time); value is the "
                        "oracle's whole-circuit fwd+bwd samples/s extrapolated from it",
                "wall_s": dt}
        print(json.dumps(line))
        return
    if args.workload != "c3":
        if rank == 0:
            run_other(args, world, rank, local)
        return
    out, wl = run_ours(args, world, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            pool = _oracle_pool(cores)
            v, _, sample, ext, _ = oracle_bounded(wl, pool, cores, per_core_s=max(1.0, 20.0 / cores))
            pool.close()
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample, **ext}
        line = json.dumps(out)
        print(line)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(line + "\n")
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
