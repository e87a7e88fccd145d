#!/usr/bin/env python3
"""Benchmark of the hierarchical merge-and-truncate rank-k SVD on GB300.

Workload (one "step" = the whole hot path once): the power-law matrix
A = U diag(s) V^T + 1e-6 N(0,1), 65536 x 65536 FP32 (17.2 GB), U, V random
orthonormal with 512 columns, s_i = (i+1)^-1.5; 64 x 64 grid of 1024 x 1024
blocks, fixed rank k = 128, column-then-row merge tree, one power step of
the block range finder.  Seeded and synthetic, generated on the device.
The timed path is the BF16-mixed one (tensor-core input products); the
plain FP32 path runs the same workload beside it ("mixed vs plain FP32").

Metric: time-to-rank-k and input GB/s (m n 4 bytes / time), measured on the
device with CUDA events around K steps (inputs resident in HBM, 17.2 GB >>
the 129 MB L2, so no flush is needed), max over ranks.

Accuracy, reported beside the time:
* on the timed 65536^2 result: certified bounds (Weyl bands around the
  planted spectrum plus Kato-Temple on the Hermitian dilation, in FP64 on the
  device) on |sigma_i - sigma_i(X)| / sigma_i for the modes well above the
  noise edge, and the error against a converged FP32 randomized SVD;
* against the FP64 oracle on the same recipe at 8192^2 (same blocks, k and
  power steps): sigma and subspace errors over the modes well above the noise
  edge (gate 1e-4 / 1e-3), the literal maximum over all k, the reconstruction
  error against the oracle's, and the paper's error ||X_k - Xhat_k||_F /
  ||X_k||_F against the truncated SVD.
That oracle run is also the CPU baseline (all host cores; plus one thread on
one row slab).

--gpus N under torchrun: every rank factors its own independent matrix of the
same configuration (no collective on the data path), value = N m n 4 / max
rank time ("weak" scaling).
--impl reference: the FP64 CPU oracle (the paper's algorithm in numpy /
LAPACK) timed on the host cores, each step one row slab of the workload.
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

M = N = 65536
BR = BC = 1024
K = 128
MODES = 512
NOISE = 1e-6
TAG = 5
ORACLE_SIZE = 8192          # the recipe at this size is compared with the oracle
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
# DRAM bytes per unit of work of the dominant kernels, from ncu captures of
# the current kernels (dram__bytes_read.sum + dram__bytes_write.sum): the
# core SVDs per core (two launches of k_jacobi_rr at 8192^2: 23.55 MB over
# 96 cores of 256 x 256); absent where no capture of the current kernel exists
TRAFFIC_PER_UNIT = {"jacobi": (16979456 + 14592 + 6555392 + 0) / 96}


def spectrum():
    return (np.arange(MODES) + 1.0) ** -1.5


def noise_edge(m, n):
    """Upper bound of the noise's spectral norm, noise (sqrt m + sqrt n) (+5%)."""
    return 1.05 * NOISE * (np.sqrt(m) + np.sqrt(n))


def workload_config(prec, q):
    mb = M * N * 4 / 1e6
    l2 = (f"input {mb:.0f} MB > 129 MB L2 (no flush needed)" if mb > 129 else
          f"input {mb:.0f} MB fits L2: profiling size only, not a bench line")
    return {"workload": f"power_law_{M}" if M == N else f"power_law_{M}x{N}", "m": M, "n": N, "block": [BR, BC],
            "grid": [M // BR, N // BC], "k": K, "spectrum": f"s_i=(i+1)^-1.5, {MODES} modes", "noise": NOISE,
            "tree": "col_then_row", "path": prec, "power_iters": q, "input_dtype": "f32", "l2": l2}


def set_size(size):
    """--size S: the same construction on an S x S matrix (same blocks, k and
    spectrum) -- small cases for profiler captures."""
    global M, N
    M = N = size


def make_input(rank=0, size=None):
    """The recipe on the host (numpy FP32) at size x size (default: the bench
    size); rank r > 0 of a multi-GPU run draws its own independent matrix of
    the same construction (seed tag 5 + 1000 r)."""
    from paper_1710_02812_gb300 import workloads as W
    s = size or M
    return W.planted(s, s, spectrum()[:min(MODES, s)], noise=NOISE, tag=TAG + 1000 * rank, dtype=np.float32)


def make_input_device(rank, device):
    """The bench matrix on the device (torch's seeded generator; the 17 GB
    FP32 matrix is never built on the host)."""
    from paper_1710_02812_gb300 import workloads as W
    return W.planted_device(M, N, spectrum()[:min(MODES, M, N)], noise=NOISE, tag=TAG + 1000 * rank,
                            device=device)


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




# ------------------------------------------------------------------ accuracy measures (torch, on the device)

def _rows(x, r0, r1, bf16):
    xb = x[r0:r1]
    return xb.to(__import__("torch").bfloat16).float() if bf16 else xb


def ritz_pairs(x, U, S, V, upto, bf16=False, chunk=4096):
    """theta_i = u_i^T X v_i and the residual eps_i of z = [u_i; v_i]/sqrt 2 for
    the dilation [[0, X], [X^T, 0]] (FP64; X read in row chunks, rounded to
    BF16 first when the path computed on BF16 values)."""
    import torch
    u = U[:, :upto].double()
    v = V[:, :upto].double()
    u = u / torch.linalg.norm(u, dim=0)
    v = v / torch.linalg.norm(v, dim=0)
    xv = torch.empty_like(u)
    xtu = torch.zeros_like(v)
    for r0 in range(0, x.shape[0], chunk):
        xb = _rows(x, r0, r0 + chunk, bf16).double()
        xv[r0:r0 + chunk] = xb @ v
        xtu += xb.t() @ u[r0:r0 + chunk]
    theta = (u * xv).sum(0)
    e1 = torch.linalg.norm(xv - u * theta, dim=0)
    e2 = torch.linalg.norm(xtu - v * theta, dim=0)
    return theta.cpu().numpy(), torch.sqrt((e1 ** 2 + e2 ** 2) / 2).cpu().numpy()


def rounding_norm_estimate(x, iters=30, chunk=4096, seed=7):
    """||bf16(X) - X||_2 by the power method on R^T R (a block of 4 vectors,
    R formed chunk by chunk, never stored): a lower estimate, used x 1.5."""
    import torch
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    q, _ = torch.linalg.qr(torch.randn((x.shape[1], 4), generator=g, device=x.device, dtype=torch.float64))
    lam = 0.0
    for _ in range(iters):
        z = torch.zeros_like(q)
        for r0 in range(0, x.shape[0], chunk):
            xb = x[r0:r0 + chunk]
            rc = (xb.to(torch.bfloat16).float() - xb).double()
            z += rc.t() @ (rc @ q)
        lam = float(torch.linalg.eigvalsh(q.t() @ z).max())
        q, _ = torch.linalg.qr(z)
    return lam ** 0.5


def certified_errors(x, U, S, V, bf16):
    """Certified |sigma_i - sigma_i(X)| / sigma_i over the planted modes with
    s_i > 10 nb (nb >= ||X - X_free||_2): Weyl bands [s_j - nb, s_j + nb] hold
    sigma_j(X); where theta_i = u_i^T X v_i lies strictly between the bands of
    its neighbours, Kato-Temple bounds |theta_i - sigma_i(X)| by
    eps_i^2 / (distance to those bands), and |sigma_i - theta_i| is added."""
    s = spectrum()
    m, n = x.shape
    nb = noise_edge(m, n) + 1e-6
    r2 = rounding_norm_estimate(x) if bf16 else 0.0
    nb += 1.5 * r2
    lead = int(np.sum(s[:S.numel()] > 10 * nb))
    theta, eps = ritz_pairs(x, U, S, V, lead, bf16=bf16)
    sig = S[:lead].double().cpu().numpy()
    free = np.concatenate([s, [0.0]])
    bound = np.full(lead, np.nan)
    for i in range(lead):
        alpha = free[i + 1] + nb
        beta = free[i - 1] - nb if i > 0 else np.inf
        delta = min(theta[i] - alpha, beta - theta[i])
        if delta > 0:
            bound[i] = (abs(sig[i] - theta[i]) + eps[i] ** 2 / delta) / sig[i]
    rq = np.abs(sig - theta) / sig
    ok = ~np.isnan(bound)
    return {"modes": lead, "certified_modes": int(ok.sum()),
            "sigma_rel_err_bound_max": float(np.nanmax(bound)) if ok.any() else None,
            "rayleigh_quotient_gap_max": float(rq.max()) if lead else None,
            "nb": nb, "rounding_norm_estimate": r2 if bf16 else None,
            "pass": bool(ok.sum() >= min(lead, 6) and (not ok.any() or np.nanmax(bound) <= 1e-4)),
            "method": "Weyl bands around the planted spectrum + Kato-Temple on the Hermitian dilation (FP64)"}


def converged_truncated_svd(x, k, q, dtype):
    """Rank-k truncation of a randomized SVD with k' = 2k and q power steps in
    `dtype` (torch, no TF32): for the power-law spectrum (s_{2k+1}/s_k)^(2q+1)
    is below 1e-12 at q >= 10, so this is the truncated SVD X_k to rounding."""
    import torch
    g = torch.Generator(device=x.device)
    g.manual_seed(11)
    xx = x.to(dtype)
    y = xx @ torch.randn((x.shape[1], 2 * k), generator=g, device=x.device, dtype=dtype)
    qy, _ = torch.linalg.qr(y)
    for _ in range(q):
        qw, _ = torch.linalg.qr(xx.t() @ qy)
        qy, _ = torch.linalg.qr(xx @ qw)
    b = qy.t() @ xx
    ub, sb, vbt = torch.linalg.svd(b, full_matrices=False)
    return (qy @ ub[:, :k]), sb[:k], vbt[:k].t()


def error_vs_truncated(Uk, Sk, Vk, U, S, V):
    """||X_k - Xhat_k||_F / ||X_k||_F from the factors (Section 4's error),
    without forming either m x n matrix."""
    import torch
    Uk, Sk, Vk, U, S, V = (t.double() for t in (Uk, Sk, Vk, U, S, V))
    cross = torch.sum((Uk.t() @ U) * ((Sk[:, None] * (Vk.t() @ V)) * S[None, :]))
    d2 = float((Sk ** 2).sum() + (S ** 2).sum() - 2 * cross)
    return max(d2, 0.0) ** 0.5 / float(torch.linalg.norm(Sk))


# ------------------------------------------------------------------ the oracle legs (host)

def oracle_run(x):
    """The FP64 oracle on a host matrix with the bench's blocks and k."""
    import oracle
    t0 = time.perf_counter()
    res = oracle.hmat_svd(x, BR, BC, oracle.Rule("fixed_k", K, rank_tol=1e-5))
    return res, time.perf_counter() - t0


def reference_sample():
    """One row slab of the bench workload's host recipe: rows 0..BR, columns
    0..min(n, 8192) (min(n, 8192) / BC blocks, the same block size and k)."""
    from paper_1710_02812_gb300 import workloads as W
    cols = min(N, ORACLE_SIZE)
    return W.planted_band(M, N, spectrum()[:min(MODES, M, N)], noise=NOISE, tag=TAG, rows=min(BR, M), cols=cols)


def one_thread_sample():
    """The reference sample through the oracle in a child process with one
    BLAS thread (the paper's single-core framing); returns (seconds, bytes) or
    None."""
    code = ("import sys; sys.path.insert(0, %r); import bench; bench.set_size(%d); "
            "x = bench.reference_sample(); r, t = bench.oracle_run(x); print(t, x.size * 4)") % (ROOT, M)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        t, b = p.stdout.strip().splitlines()[-1].split()
        return float(t), int(b)
    except Exception:
        return None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    """The oracle as it stands, timed on the host cores: each step factors one
    row slab (BR rows x min(n, 8192) columns) of the recipe."""
    if rank != 0:
        return 0
    x = reference_sample()
    rows, cols = x.shape
    for _ in range(args.warmup):
        oracle_run(x)
    times = [oracle_run(x)[1] for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    val = x.size * 4 / (ms * 1e-3) / 1e9
    sample = (f"one row slab, {rows} x {cols}, of the workload's host recipe ({cols // BC} blocks, same block "
              f"size and k; the {M}x{N} matrix has {(M // BR) * (N // BC)} blocks)")
    line = {"impl": "reference", "metric": "input GB/s (rank-k SVD, top-k sigma rel err <= 1e-4)",
            "value": val, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config("oracle_f64", 0),
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ the GPU leg

def device_factors(plan, dev):
    import torch
    k = plan.kcap
    U = torch.empty((k, plan.m[0]), dtype=torch.float32, device=dev)
    S = torch.empty(k, dtype=torch.float32, device=dev)
    V = torch.empty((k, plan.n[0]), dtype=torch.float32, device=dev)
    r = plan.factors_device(U, S, V, 0)
    return U[:r].t(), S[:r], V[:r].t()


def timed_steps(plan, xd, steps, stream, world, dev, sampler=None):
    import torch
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.run([xd], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    return e0.elapsed_time(e1) / steps


def oracle_parity(prec, q, dev):
    """The bench recipe at ORACLE_SIZE^2 (same blocks, k, power steps): the
    GPU path and the FP64 oracle on the same values (BF16-rounded for the
    mixed path), plus the paper's error against the truncated SVD of X.  Also
    returns the oracle's time on the full-precision input (the CPU baseline)."""
    import torch
    import oracle
    from paper_1710_02812_gb300 import hsvd
    from paper_1710_02812_gb300 import workloads as W
    size = min(ORACLE_SIZE, M)
    x = make_input(0, size)
    xd = torch.from_numpy(x).to(dev)
    uk, sk, vk = converged_truncated_svd(xd, K, 12, torch.float64)
    res_fp32, t_oracle = oracle_run(x.astype(np.float64))
    out = {}
    nb = noise_edge(size, size)
    s = spectrum()
    gate = int(np.sum(s[:K] > 10 * nb))
    for path in ("bf16_mixed", "f32"):
        plan = hsvd.Plan(size, size, BR, BC, "fixed_k", K, prec=path, power_iters=q)
        plan.run([xd])
        u, sg, v = plan.factors(0)
        U, S, V = device_factors(plan, dev)
        st = plan.status()
        plan.close()
        ref = res_fp32 if path == "f32" else oracle_run(W.bf16_round(x).astype(np.float64))[0]
        lit = oracle.sigma_rel_err(sg, ref.s, min(K, sg.size, ref.s.size))
        xx = x.astype(np.float64) if path == "f32" else W.bf16_round(x).astype(np.float64)
        nx = np.linalg.norm(xx)
        rg = np.linalg.norm(xx - (u.astype(np.float64) * sg) @ v.T.astype(np.float64)) / nx
        ro = np.linalg.norm(xx - (ref.u * ref.s) @ ref.v.T) / nx
        d = {"modes_gated": gate, "gate_rule": f"planted s_i > 10 noise (2 sqrt {size})",
             "sigma_rel_err_gated": oracle.sigma_rel_err(sg, ref.s, gate),
             "subspace_angle_u_gated": oracle.leading_subspace_angle(u, ref.u, ref.s, upto=gate),
             "subspace_angle_v_gated": oracle.leading_subspace_angle(v, ref.v, ref.s, upto=gate),
             "sigma_rel_err_all_k_literal": lit,
             "sigma_normwise_all_k": float(np.max(np.abs(sg - ref.s)) / ref.s[0]),
             "recon_err": float(rg), "recon_err_oracle": float(ro),
             "err_vs_truncated_svd": error_vs_truncated(uk, sk, vk, U, S, V),
             "oracle_err_vs_truncated_svd": error_vs_truncated(
                 uk, sk, vk, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ref.u, ref.s, ref.v))),
             "rank": int(sg.size), "status": st}
        d["pass"] = bool(d["sigma_rel_err_gated"] <= 1e-4 and d["subspace_angle_u_gated"] <= 1e-3 and
                         d["subspace_angle_v_gated"] <= 1e-3 and abs(rg - ro) <= 0.01 * ro + 50 * 6e-8)
        if path == "bf16_mixed":
            d["reference"] = "oracle on the same BF16-rounded values"
            d["vs_fp32_input"] = {"sigma_rel_err_gated": oracle.sigma_rel_err(sg, res_fp32.s, gate),
                                  "subspace_angle_u_gated": oracle.leading_subspace_angle(u, res_fp32.u, res_fp32.s,
                                                                                          upto=gate)}
        out[path] = d
    out["truncated_svd"] = "rank-k truncation of an FP64 randomized SVD with 12 power steps (converged)"
    out["size"] = [size, size]
    return out, t_oracle, size * size * 4


def run_ours(args, world, rank, local):
    import torch
    from paper_1710_02812_gb300 import hsvd
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local)
    torch.backends.cuda.matmul.allow_tf32 = False
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    q = args.power_iters
    xd = make_input_device(rank, dev)
    torch.cuda.synchronize(dev)

    # ---- the timed path: warm-up, then K steps with CUDA events around the
    # core-SVD (Jacobi) launches inside the replayed graph (the dominant
    # family's live time); the per-family split comes from an instrumented
    # pass after the timed region
    plan = hsvd.Plan(M, N, BR, BC, "fixed_k", K, prec=args.prec, power_iters=q, host_staging=True,
                     autotune=not args.no_autotune)
    for _ in range(args.warmup):
        plan.run([xd], stream=stream)
    torch.cuda.synchronize(dev)
    plan.set_timing(2)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ms = timed_steps(plan, xd, args.steps, stream, world, dev)
    clocks = sampler.stop()
    ms = reduce_max(world, ms, dev)
    jac_ms, jac_runs = plan.step_times()
    plan.set_timing(1)
    for _ in range(0 if args.quick else 2):
        plan.run([xd], stream=stream)
    step_ms, runs = plan.step_times()
    plan.set_timing(False)
    steps = plan.steps()
    st = plan.status()
    workspace = plan.workspace_bytes
    accuracy_full = None
    if rank == 0 and not args.no_oracle:
        plan.run([xd], stream=stream)
        U, S, V = device_factors(plan, dev)
        accuracy_full = certified_errors(xd, U, S, V, bf16=args.prec == "bf16_mixed")
        uk, sk, vk = converged_truncated_svd(xd, K, 6, torch.float32)
        accuracy_full["err_vs_truncated_svd"] = error_vs_truncated(uk, sk, vk, U, S, V)
        accuracy_full["truncated_svd"] = "rank-k truncation of an FP32 randomized SVD, k' = 2k, 6 power steps"
        del U, S, V, uk, sk, vk

    # ---- end to end through the C ABI with host buffers: pinned input read by
    # hsvd_run_host, factors copied back to the host every step
    e2e_ms = float("nan")
    if not args.quick:
        xh = torch.empty((M, N), dtype=torch.float32, pin_memory=True)
        xh.copy_(xd)
        for _ in range(max(1, args.warmup // 2)):
            plan.run_host([xh], stream=stream)
            plan.factors(0, stream=stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.run_host([xh], stream=stream)
            plan.factors(0, stream=stream)
        e2e_ms = 1e3 * (time.perf_counter() - t0) / args.steps
        e2e_ms = reduce_max(world, e2e_ms, dev)
        del xh
    h2d = M * N * 4
    d2h = (M + N) * plan.kcap * 4 + plan.kcap * 4 + 4
    launches = plan.launches_per_run
    tuned = {}
    for name, chosen, cnt in plan.variants():
        if cnt > 1:
            tuned[chosen] = tuned.get(chosen, 0) + 1
    plan.close()
    del plan
    torch.cuda.empty_cache()

    # ---- roofline of the dominant kernel family (device time per run)
    fam = {}
    for info, t in zip(steps, step_ms):
        f = fam.setdefault(info["kind"], {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
        f["ms"] += t / max(1, runs)
        f["flops"] += info["flops"]
        f["bytes"] += info["bytes"]
        f["launches"] += 1
    if runs == 0:  # --quick: no per-step pass; the live core-SVD times only
        for f in fam.values():
            f["ms"] = 0.0
        fam.setdefault("jacobi", {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
    dom = "jacobi" if runs == 0 else max(fam, key=lambda k: fam[k]["ms"])
    pk, pk_src = peaks()
    d = fam[dom]
    jac_live = sum(t for info, t in zip(steps, jac_ms) if info["kind"] == "jacobi") / max(1, jac_runs)
    traffic = TRAFFIC_PER_UNIT.get(dom)
    if dom == "jacobi":
        d = dict(d, ms=jac_live)          # the timed region's own events
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"kernel": "k_jacobi_* (one-sided Jacobi core SVDs)", "bound": "alu", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "work": "22 n^3 flops per n x n core (Section 3.1 count)"}
    elif dom == "gemm_tc":
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"kernel": "k_tc_gemm (tcgen05 BF16)", "bound": "tensor", "achieved": achieved,
                "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                "frac": achieved / pk["bf16_tflops_sustained"], "peak_source": pk_src + " (bf16 sustained)"}
    elif dom in ("gemm_nn", "gemm_tn", "convert", "signs"):
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        roof = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "peak_source": pk_src,
                "work": "operands read once + result written once"}
    else:
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        roof = {"kernel": f"k_{dom}", "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "peak_source": "derived FP32 peak",
                "work": "k^3 flops per k x k factorisation and inverse"}
    # per launch, like achieved: the family's units (cores) per launch x bytes per unit
    roof["traffic"] = (traffic * st["jacobi_cores"] / max(1, d["launches"])
                       if traffic and dom == "jacobi" else None)
    if roof["traffic"] is not None:
        roof["traffic_source"] = "ncu DRAM bytes per core (k_jacobi_rr, 8192^2 capture) x cores per launch"
    roof["share_of_step"] = d["ms"] / ms
    roof["launches_per_step"] = d["launches"]
    roof["ms_per_step"] = d["ms"]
    roof["timing"] = ("CUDA events around each launch of the family inside the timed region"
                      if dom == "jacobi" else "instrumented pass (events around every step)")

    # ---- the other side of "mixed vs plain FP32": same workload, FP32 path
    compare = None
    if not args.no_compare and args.prec != "f32":
        pf = hsvd.Plan(M, N, BR, BC, "fixed_k", K, prec="f32", power_iters=q, autotune=not args.no_autotune)
        for _ in range(args.warmup):
            pf.run([xd], stream=stream)
        torch.cuda.synchronize(dev)
        fms = reduce_max(world, timed_steps(pf, xd, args.steps, stream, world, dev), dev)
        facc = None
        if rank == 0 and not args.no_oracle:
            U, S, V = device_factors(pf, dev)
            facc = certified_errors(xd, U, S, V, bf16=False)
            del U, S, V
        compare = {"path": "f32", "ms_per_step": fms, "value": world * M * N * 4 / (fms * 1e-3) / 1e9,
                   "unit": "GB/s", "speedup_of_headline": fms / ms, "certified_accuracy": facc,
                   "workspace_bytes": pf.workspace_bytes}
        pf.close()
        del pf
        torch.cuda.empty_cache()

    # ---- accuracy against the oracle on the same recipe at 8192^2, which is
    # also the CPU baseline (the oracle as it stands, all host cores)
    parity = cpu_base = None
    if rank == 0 and not args.no_oracle:
        del xd
        torch.cuda.empty_cache()
        parity, t_oracle, ob = oracle_parity(args.prec, q, dev)
        cpu_base = {"value": ob / t_oracle / 1e9, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                    "sample": f"the workload's recipe at {parity['size'][0]}^2 (same block size, k and spectrum; "
                              f"{(parity['size'][0] // BR) ** 2} of the {(M // BR) * (N // BC)} blocks), one run, "
                              f"{t_oracle:.1f} s, numpy/LAPACK FP64"}
        one = one_thread_sample()
        if one:
            cpu_base["one_thread"] = {"value": one[1] / one[0] / 1e9, "unit": "GB/s", "cores": 1,
                                      "sample": f"one row slab ({one[1] // 4 // min(N, ORACLE_SIZE)} x "
                                                f"{min(N, ORACLE_SIZE)}) of the workload, {one[0]:.1f} s"}

    value = world * M * N * 4 / (ms * 1e-3) / 1e9
    line = {"metric": "input GB/s (rank-k SVD, top-k sigma rel err <= 1e-4)", "value": value, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "time_to_rank_k_ms": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "bf16_mixed": "bf16"}[args.prec], "data": "synthetic",
            "config": dict(workload_config(args.prec, q),
                           autotuned={"on": not args.no_autotune, "launches_by_choice": tuned}),
            "roofline": roof,
            "kernel_families_ms": {k: round(v["ms"], 4) for k, v in sorted(fam.items(), key=lambda kv: -kv[1]["ms"])},
            "kernel_families_note": "instrumented pass after the timed region: events around every step",
            "e2e": {"value": world * M * N * 4 / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
            "accuracy_certified": accuracy_full,
            "accuracy_vs_oracle": parity,
            "plain_fp32": compare,
            "status": st,
            "workspace_bytes": workspace,
            "cpu_baseline": cpu_base}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_split_rows(args, world, rank, local):
    """--split rows: ONE matrix of the workload over the ranks, each holding a
    band of whole row slabs (rowsplit.factor_rows: band plans, the merge tree
    over ranks by point-to-point factor sends, V_hat broadcast, CholeskyQR2
    of the recovery with the Grams summed over the bands).  value = m n 4 /
    max rank time ("strong" scaling: the total work is fixed)."""
    import torch
    from paper_1710_02812_gb300 import rowsplit
    from paper_1710_02812_gb300 import workloads as W
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local)
    torch.backends.cuda.matmul.allow_tf32 = False
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    q = args.power_iters
    row0, rows = rowsplit.band_rows(M, BR, world)[rank]
    xb = W.planted_device(M, N, spectrum()[:min(MODES, M, N)], noise=NOISE, tag=TAG, device=dev,
                          rows=(row0, row0 + rows))
    band = rowsplit.DeviceBand(xb, N, row0, BR, BC, K, prec=args.prec, power_iters=q)
    comm = rowsplit.TorchComm() if world > 1 else rowsplit.SingleComm()
    for _ in range(args.warmup):
        rowsplit.factor_rows(band, comm)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        u, s, v = rowsplit.factor_rows(band, comm)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop()
    ms = reduce_max(world, e0.elapsed_time(e1) / args.steps, dev)
    # end to end: this rank's band from page-locked host memory, the factors
    # (its U rows, S, V) back to the host every step
    xh = torch.empty((rows, N), dtype=torch.float32, pin_memory=True)
    xh.copy_(xb)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xb.copy_(xh, non_blocking=True)
        u, s, v = rowsplit.factor_rows(band, comm)
        u, s, v = u.cpu(), s.cpu(), v.cpu()
    e2e_ms = reduce_max(world, 1e3 * (time.perf_counter() - t0) / args.steps, dev)
    st = band.plan.status()
    value = M * N * 4 / (ms * 1e-3) / 1e9
    line = {"metric": "input GB/s (rank-k SVD, top-k sigma rel err <= 1e-4)", "value": value, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "time_to_rank_k_ms": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": {"f32": "f32", "bf16_mixed": "bf16"}[args.prec], "data": "synthetic",
            "config": dict(workload_config(args.prec, q), split="rows", bands=rowsplit.band_rows(M, BR, world)),
            "e2e": {"value": M * N * 4 / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": rows * N * 4, "d2h_bytes_per_step": (rows + N + 1) * band.kc * 4,
                    "ms_per_step": e2e_ms},
            "gpu_launches": None, "clocks": clocks, "status": st, "roofline": None, "cpu_baseline": None,
            "note": "one matrix split by row bands; the roofline and CPU baseline are on the default single-"
                    "matrix line"}
    band.close()
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
    ap.add_argument("--no-oracle", action="store_true", help="skip the accuracy measures and the CPU baseline")
    ap.add_argument("--no-autotune", dest="no_autotune", action="store_true",
                    help="default kernels instead of the autotuner's choices (timed on the first warm-up run)")
    ap.add_argument("--quick", action="store_true",
                    help="the timed steps only (no accuracy, CPU baseline, comparison, end-to-end or per-step "
                         "pass): for profiler launch lists")
    ap.add_argument("--split", default="none", choices=["none", "rows"],
                    help="rows: one matrix over the ranks by row bands (strong scaling); "
                         "none: every rank its own matrix (weak scaling)")
    ap.add_argument("--size", type=int, default=65536,
                    help="matrix size (default 65536, the bench workload; smaller sizes are for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.quick:
        args.no_oracle = args.no_compare = True
    if args.size != 65536:
        if args.size < BR or args.size % BR:
            ap.error(f"--size must be a multiple of the {BR}-row block")
        set_size(args.size)
    world, rank, local = dist_init()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        if args.split == "rows":
            return run_split_rows(args, world, rank, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
