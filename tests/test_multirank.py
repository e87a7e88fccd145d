"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards by independent problems: under torchrun every rank factors
its own matrix of the bench construction with no collective on the data
path; the ranks meet only at the barriers around the timed region and in
the max-over-ranks of the step time.  These tests run that host logic in two
CPU processes: the barrier and MAX reduction, the per-rank inputs, and the
reference arm (rank 0 alone runs and prints; the other ranks exit 0).
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank: int, world: int, port: int) -> dict:
    env = dict(os.environ)
    env.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return env


HELPERS = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import bench
    bench.set_size(1024)
    world, rank, local = bench.dist_init()
    bench.barrier(world)
    mx = bench.reduce_max(world, 1.5 + rank, "cpu")
    x = bench.make_input(rank)
    x0 = bench.make_input(0)
    print(json.dumps({{"rank": rank, "world": world, "max": mx, "sum": float(np.float64(x).sum()),
                      "same_as_rank0": bool(np.array_equal(x, x0)), "shape": list(x.shape)}}))
    bench.barrier(world)
    import torch.distributed as dist
    dist.destroy_process_group()
""")


def test_barrier_max_and_per_rank_inputs_gloo():
    port = _free_port()
    code = HELPERS.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["world"] for d in outs] == [2, 2]
    # max over ranks is the larger of the two step times, on every rank
    assert [d["max"] for d in outs] == [2.5, 2.5]
    # rank 0 keeps the bench matrix; rank 1 draws its own of the same shape
    assert outs[0]["same_as_rank0"] and not outs[1]["same_as_rank0"]
    assert outs[0]["shape"] == outs[1]["shape"] == [1024, 1024]
    assert outs[0]["sum"] != outs[1]["sum"]


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched the way the multi-GPU bench is:
    rank 0 times the oracle and prints the one JSON line, rank 1 exits 0."""
    port = _free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--size", "1024", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["m"] == d["config"]["n"] == 1024
