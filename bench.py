#!/usr/bin/env python3
"""Benchmark of the hierarchical merge-and-truncate rank-k SVD on GB300.

Workload (one "step" = the whole hot path once): an 8192 x 8192 FP32 matrix
A = U diag(s) V^T + 1e-5 N(0,1), U, V random orthonormal with 512 columns,
s_i = exp(-i/20); 16 x 16 grid of 512 x 512 blocks, fixed rank k = 64,
column-then-row merge tree.  Inputs are seeded and synthetic.

Metric: time-to-rank-k and input GB/s (m n 4 bytes / time), measured on the
device with CUDA events around K steps (inputs resident in HBM, 268 MB > the
129 MB L2, so no flush is needed), max over ranks.  The top-k singular values
are checked against the FP64 oracle (relative error <= 1e-4).

--gpus N under torchrun: every rank factors its own independent matrix of the
same configuration (the path shards by independent problems: no collective
on the data path), value = N m n 4 / max rank time ("weak" scaling).
--impl reference: the FP64 CPU oracle (the paper's algorithm in numpy /
LAPACK) timed on the host cores on a row-band sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = 8192
BR = BC = 512
K = 64
MODES = 512
NOISE = 1e-5
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
# DRAM bytes per 128 x 128 core of k_jacobi_bp (ncu dram__bytes_read + dram__bytes_write of one
# merge-level launch of the 2048^2 case: 472576 bytes for 8 cores)
JACOBI_DRAM_BYTES_PER_CORE = 472576 / 8


def workload_config(prec, q):
    mb = M * N * 4 / 1e6
    l2 = (f"input {mb:.0f} MB > 129 MB L2 (no flush needed)" if mb > 129 else
          f"input {mb:.0f} MB fits L2: profiling size only, not a bench line")
    return {"workload": f"exp_decay_{M}" if M == N else f"exp_decay_{M}x{N}", "m": M, "n": N, "block": [BR, BC],
            "grid": [M // BR, N // BC], "k": K, "spectrum": f"s_i=exp(-i/20), {MODES} modes", "noise": NOISE,
            "tree": "col_then_row", "path": prec, "power_iters": q, "input_dtype": "f32", "l2": l2}


def set_size(size):
    """--size S: the same construction on an S x S matrix (same blocks, k and
    spectrum) -- small cases for profiler captures."""
    global M, N, MODES
    M = N = size
    MODES = min(512, size)


def make_input(rank=0):
    """The bench matrix; rank r > 0 of a multi-GPU run draws its own
    independent matrix of the same construction (seed tag 2 + 1000 r)."""
    from paper_1710_02812_gb300 import workloads as W
    return W.exp_decay(M, N, MODES, NOISE, tag=2 + 1000 * rank, dtype=np.float32)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_run(x, rows=None):
    """The FP64 oracle on the full matrix or on its first `rows` rows."""
    import oracle
    xs = x if rows is None else x[:rows]
    t0 = time.perf_counter()
    res = oracle.hmat_svd(xs, BR, BC, oracle.Rule("fixed_k", K, rank_tol=1e-5))
    return res, time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    x = make_input()
    rows = min(2048, M)  # row band: 4 of the 16 slabs, every block / merge step of the path
    for _ in range(args.warmup):
        oracle_run(x, rows)
    times = []
    for _ in range(args.steps):
        times.append(oracle_run(x, rows)[1])
    ms = 1e3 * sum(times) / len(times)
    val = rows * N * 4 / (ms * 1e-3) / 1e9
    sample = f"rows 0..{rows} of the {M}x{N} matrix ({rows // BR} of {M // BR} row slabs, same grid and k)"
    line = {"impl": "reference", "metric": "input GB/s (rank-k SVD, top-k sigma rel err <= 1e-4)",
            "value": val, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config("oracle_f64", 0),
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, world, rank, local):
    import torch
    import oracle
    from paper_1710_02812_gb300 import hsvd
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    x = make_input(rank)
    xd = torch.from_numpy(x).to(dev)
    q = args.power_iters
    plan = hsvd.Plan(M, N, BR, BC, "fixed_k", K, prec=args.prec, power_iters=q, host_staging=True)
    stream = torch.cuda.current_stream(dev)

    # ---- accuracy gate against the oracle (rank 0; also the CPU baseline)
    accuracy = None
    cpu_base = None
    if rank == 0 and not args.no_oracle:
        plan.run([xd])
        u, s, v = plan.factors(0)
        res, t_oracle = oracle_run(x)
        ref_s, ref_u = res.s, res.u
        if args.prec == "bf16_mixed":
            # the mixed path computes on the BF16-rounded input: the gate is
            # against the oracle on those same values (storage rounding is not
            # method error); the error against the FP32 input is reported too
            from paper_1710_02812_gb300 import workloads as W
            gres, _ = oracle_run(W.bf16_round(x))
        else:
            gres = res
        err = oracle.sigma_rel_err(s, gres.s, K)
        ang = oracle.leading_subspace_angle(u, gres.u, gres.s, upto=K)
        accuracy = {"sigma_rel_err_max": err, "subspace_angle_max": ang, "rank": int(s.size),
                    "gate_sigma": 1e-4, "gate_angle": 1e-3,
                    "pass": bool(err <= 1e-4 and ang <= 1e-3 and s.size == K),
                    "reference": "oracle on the same (BF16-rounded) input" if args.prec == "bf16_mixed" else "oracle"}
        if args.prec == "bf16_mixed":
            accuracy["vs_fp32_input"] = {"sigma_rel_err_max": oracle.sigma_rel_err(s, res.s, K),
                                         "subspace_angle_max": oracle.leading_subspace_angle(u, res.u, res.s, upto=K)}
        cpu_base = {"value": M * N * 4 / t_oracle / 1e9, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                    "sample": f"full {M}x{N} matrix, 1 run ({t_oracle:.1f} s, numpy/LAPACK FP64)"}

    # ---- warm-up, then K timed steps; CUDA events around the core-SVD
    # (Jacobi) launches only, the dominant family, inside the timed region
    # (events around every step add ~1 ms per step: the per-family split is
    # taken in a separate instrumented pass below)
    for _ in range(args.warmup):
        plan.run([xd])
    torch.cuda.synchronize(dev)
    plan.set_timing(2)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run([xd], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = reduce_max(world, ms, dev)
    jac_ms, jac_runs = plan.step_times()
    plan.set_timing(1)                       # instrumented pass: every step
    for _ in range(min(args.steps, 5)):
        plan.run([xd], stream=stream)
    step_ms, runs = plan.step_times()
    plan.set_timing(False)
    steps = plan.steps()
    st = plan.status()

    # ---- end to end through the C ABI with host buffers (pinned input)
    xh = torch.from_numpy(x).pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        plan.run_host([xh], stream=stream)
        plan.factors(0, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.run_host([xh], stream=stream)
        u_h, s_h, v_h = plan.factors(0, stream=stream)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
    e2e_ms = reduce_max(world, e2e_ms, dev)
    h2d = M * N * 4
    d2h = (M + N) * plan.kcap * 4 + plan.kcap * 4 + 4

    # ---- roofline of the dominant kernel family (device time per run)
    fam = {}
    for info, t in zip(steps, step_ms):
        f = fam.setdefault(info["kind"], {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
        f["ms"] += t / max(1, runs)
        f["flops"] += info["flops"]
        f["bytes"] += info["bytes"]
        f["launches"] += 1
    dom = max(fam, key=lambda k: fam[k]["ms"])
    pk, pk_src = peaks()
    d = fam[dom]
    jac_live = sum(t for info, t in zip(steps, jac_ms) if info["kind"] == "jacobi") / max(1, jac_runs)
    if dom == "jacobi":
        d = dict(d, ms=jac_live)          # the timed region's own events
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"kernel": "k_jacobi (one-sided Jacobi core SVD)", "bound": "alu", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": JACOBI_DRAM_BYTES_PER_CORE * st["jacobi_cores"] / max(1, d["launches"]),
                "traffic_source": "ncu DRAM bytes per core (2048^2 merge level) x cores per launch",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "work": "22 n^3 flops per n x n core (Section 3.1 count)"}
    elif dom == "gemm_tc":
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"kernel": "k_tc_gemm (tcgen05 BF16)", "bound": "tensor", "achieved": achieved,
                "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops_sustained"],
                "traffic": None, "peak_source": pk_src + " (bf16 sustained)"}
    elif dom in ("gemm_nn", "gemm_tn"):
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        roof = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": pk_src,
                "work": "operands read once + result written once"}
    else:
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "peak_source": "derived FP32 peak"}
    roof["share_of_step"] = d["ms"] / ms
    roof["launches_per_step"] = d["launches"]
    roof["timing"] = ("CUDA events around each launch of the family inside the timed region"
                      if dom == "jacobi" else "instrumented pass (events around every step)")

    # ---- the other side of "mixed vs plain FP32": same workload, FP32 path
    compare = None
    if not args.no_compare and args.prec != "f32":
        pf = hsvd.Plan(M, N, BR, BC, "fixed_k", K, prec="f32", power_iters=q)
        for _ in range(args.warmup):
            pf.run([xd], stream=stream)
        torch.cuda.synchronize(dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            pf.run([xd], stream=stream)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        fms = c0.elapsed_time(c1) / args.steps
        facc = None
        if accuracy is not None:
            uf, sf, vf = pf.factors(0)
            facc = {"sigma_rel_err_max": oracle.sigma_rel_err(sf, ref_s, K),
                    "subspace_angle_max": oracle.leading_subspace_angle(uf, ref_u, ref_s, upto=K)}
        compare = {"path": "f32", "ms_per_step": fms, "value": world * M * N * 4 / (fms * 1e-3) / 1e9,
                   "unit": "GB/s", "speedup_of_headline": fms / ms, "accuracy_vs_oracle": facc}
        pf.close()

    value = world * M * N * 4 / (ms * 1e-3) / 1e9
    line = {"metric": "input GB/s (rank-k SVD, top-k sigma rel err <= 1e-4)", "value": value, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "time_to_rank_k_ms": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "bf16_mixed": "bf16", "f64": "f64"}[args.prec], "data": "synthetic",
            "config": workload_config(args.prec, q),
            "roofline": roof,
            "kernel_families_ms": {k: round(v["ms"], 4) for k, v in sorted(fam.items(), key=lambda kv: -kv[1]["ms"])},
            "kernel_families_note": "instrumented pass after the timed region: events around every step",
            "e2e": {"value": world * M * N * 4 / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": plan.launches_per_run * args.steps,
            "clocks": clocks,
            "accuracy_vs_oracle": accuracy,
            "plain_fp32": compare,
            "status": st,
            "cpu_baseline": cpu_base}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16_mixed", choices=["f32", "bf16_mixed"],
                    help="path timed: the BF16-mixed headline or the plain FP32 path (the metric compares the two)")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP32 comparison run")
    ap.add_argument("--power-iters", dest="power_iters", type=int, default=1)
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--size", type=int, default=8192,
                    help="matrix size (default 8192, the bench workload; smaller sizes are for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.size != 8192:
        if args.size < BR or args.size % BR:
            ap.error(f"--size must be a multiple of the {BR}-row block")
        set_size(args.size)
    world, rank, local = dist_init()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
