"""One matrix factored by several ranks, split by row bands.

The blocks of a row slab, its column MAT tree and its slab step use no other
slab, and the row MAT tree meets other slabs only at its merges (Section 3.1
of the paper: the block SVDs and the merges of each level are independent).
So each rank takes a contiguous band of whole row slabs and:

1. factors its band up to the root of its own row tree (a band plan:
   hsvd_plan with stop_after_rows, then hsvd_run and hsvd_tree_root);
2. the roots meet along a binary tree over the ranks: at level l, rank r
   (a multiple of 2^(l+1)) receives rank r + 2^l's root (V, Sigma: one
   n x k factor) and merges it with its own (hsvd_merge_run).  The tree is
   the paper's DoMergeOfSlices over the ranks (adjacent pairs, odd last
   carried); with 2^L slabs per rank the whole tree is the paper's tree over
   the slabs;
3. rank 0 sends V_hat to every rank; U is recovered from SVD(X V_hat) by
   CholeskyQR2 over the bands (hsvd_recover_*): the ranks sum two k x k
   Grams and agree on the sign of every column through a maximum and a
   minimum over k values.

Messages: log2(world) point-to-point factors of n x k, one broadcast of the
same size, and four reductions of k or k^2 values.  The computing is the
library's; this module holds the exchange schedule and moves the data with
whatever communicator it is given (torch.distributed in practice).
"""
from __future__ import annotations

from typing import List, Tuple


def band_rows(m: int, block_rows: int, world: int) -> List[Tuple[int, int]]:
    """(first row, rows) of each rank's band: the ceil(m / block_rows) row
    slabs shared out in contiguous runs, the first (slabs mod world) ranks
    taking one slab more; the last slab may be ragged.  Every rank needs a
    slab: world may not exceed the slab count."""
    if m < 1 or block_rows < 1 or world < 1:
        raise ValueError("m, block_rows and world must be positive")
    slabs = (m + block_rows - 1) // block_rows
    if world > slabs:
        raise ValueError(f"{world} ranks for {slabs} row slabs: every rank needs a slab")
    out, s0 = [], 0
    for r in range(world):
        cnt = slabs // world + (1 if r < slabs % world else 0)
        row0 = min(m, s0 * block_rows)
        row1 = min(m, (s0 + cnt) * block_rows)
        out.append((row0, row1 - row0))
        s0 += cnt
    return out


def merge_schedule(world: int) -> List[List[Tuple[int, int]]]:
    """Levels of the binary tree over the ranks: at level l the pairs
    (receiver r, sender r + 2^l) for every r that is a multiple of 2^(l+1)
    with a sender; an unpaired rank is carried.  This is DoMergeOfSlices
    (adjacent pairs, odd last carried) on the list of ranks."""
    if world < 1:
        raise ValueError("world must be positive")
    levels, step = [], 1
    while step < world:
        levels.append([(r, r + step) for r in range(0, world, 2 * step) if r + step < world])
        step *= 2
    return levels


def factor_rows(band, comm):
    """Run the row-split schedule for this rank.

    band: this rank's computing side (see DeviceBand) with methods
      local_root() -> packet, empty_packet(), merge(packet, packet) -> packet,
      recover_begin(packet) -> G, recover_orth(Gsum) -> G2,
      recover_core(G2sum) -> absmax, recover_signs(absmax_all) -> key,
      recover_finish(key_min), factors() -> (U_band, S, V).
    comm: rank, world, send(t, dst), recv(t, src), broadcast(t, src),
      all_reduce(t, op) with op in {"sum", "max", "min"} (in place).
    Returns band.factors(): this band's rows of U, and S, V (every rank)."""
    rank, world = comm.rank, comm.world
    pkt = band.local_root()
    for level in merge_schedule(world):
        for recv, send in level:
            if rank == send:
                comm.send(pkt, recv)
            elif rank == recv:
                other = band.empty_packet()
                comm.recv(other, send)
                pkt = band.merge(pkt, other)
    comm.broadcast(pkt, 0)
    g = band.recover_begin(pkt)
    comm.all_reduce(g, "sum")
    g2 = band.recover_orth(g)
    comm.all_reduce(g2, "sum")
    amax = band.recover_core(g2)
    comm.all_reduce(amax, "max")
    key = band.recover_signs(amax)
    comm.all_reduce(key, "min")
    band.recover_finish(key)
    return band.factors()


class SingleComm:
    """comm of a single rank: nothing to exchange."""

    rank, world = 0, 1

    def send(self, t, dst):
        raise RuntimeError("a single rank sends nothing")

    recv = send

    def broadcast(self, t, src):
        pass

    def all_reduce(self, t, op):
        pass


class TorchComm:
    """comm for factor_rows over torch.distributed (NCCL for CUDA tensors,
    gloo for host tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def send(self, t, dst):
        self.dist.send(t, dst, group=self.group)

    def recv(self, t, src):
        self.dist.recv(t, src, group=self.group)

    def broadcast(self, t, src):
        self.dist.broadcast(t, src, group=self.group)

    def all_reduce(self, t, op):
        ops = {"sum": self.dist.ReduceOp.SUM, "max": self.dist.ReduceOp.MAX, "min": self.dist.ReduceOp.MIN}
        self.dist.all_reduce(t, op=ops[op], group=self.group)


class DeviceBand:
    """This rank's band on its GPU: a band plan over rows [row0, row0 + rows)
    of an m x n matrix (the device tensor `x_band`), a merge plan of height n
    and the small exchange buffers.  A packet is one device tensor of
    n kcap + kcap + 1 values: V (column-major n x kcap), Sigma, the rank."""

    def __init__(self, x_band, n, row0, block_rows, block_cols, k, prec="f32", power_iters=0, in_dtype=None):
        import torch
        from . import hsvd
        self.hsvd, self.torch = hsvd, torch
        self.x, self.n, self.row0 = x_band, int(n), int(row0)
        self.rows = int(x_band.shape[0])
        self.plan = hsvd.Plan(self.rows, self.n, block_rows, block_cols, "fixed_k", k, prec=prec,
                              in_dtype=in_dtype, power_iters=power_iters, stop_after_rows=True)
        self.merger = hsvd.MergePlan(self.n, "fixed_k", k, prec=prec)
        self.kc = self.plan.kcap
        self.dt = torch.float64 if prec == "f64" else torch.float32
        dev = x_band.device
        self.dev = dev
        self.G = torch.zeros(self.kc * self.kc, dtype=self.dt, device=dev)
        self.G2 = torch.zeros_like(self.G)
        self.amax = torch.zeros(self.kc, dtype=self.dt, device=dev)
        self.key = torch.zeros(self.kc, dtype=torch.int64, device=dev)

    def _packet_parts(self, pkt):
        nk = self.n * self.kc
        return pkt[:nk], pkt[nk:nk + self.kc], pkt[nk + self.kc:]

    def empty_packet(self):
        return self.torch.zeros(self.n * self.kc + self.kc + 1, dtype=self.dt, device=self.dev)

    def _pack(self, source):
        pkt = self.empty_packet()
        V, S, R = self._packet_parts(pkt)
        r = source.tree_root(V, S) if isinstance(source, self.hsvd.Plan) else source.root(V, S)
        R.fill_(float(r))
        return pkt

    def local_root(self):
        self.plan.run([self.x])
        return self._pack(self.plan)

    def merge(self, a, b):
        Va, Sa, Ra = self._packet_parts(a)
        Vb, Sb, Rb = self._packet_parts(b)
        self.merger.run(Va, Sa, int(Ra.item()), Vb, Sb, int(Rb.item()))
        return self._pack(self.merger)

    def recover_begin(self, pkt):
        V, _, R = self._packet_parts(pkt)
        self.plan.recover_begin(V, int(R.item()), self.G)
        return self.G

    def recover_orth(self, gsum):
        self.plan.recover_orth(gsum, self.G2)
        return self.G2

    def recover_core(self, g2sum):
        self.plan.recover_core(g2sum, self.amax)
        return self.amax

    def recover_signs(self, amax_all):
        self.plan.recover_signs(amax_all, self.row0, self.key)
        return self.key

    def recover_finish(self, key_min):
        self.plan.recover_finish(key_min)

    def factors(self):
        """(U rows of this band (rows x r), S (r), V (n x r)), device tensors."""
        kc, torch = self.kc, self.torch
        U = torch.empty((kc, self.rows), dtype=self.dt, device=self.dev)
        S = torch.empty(kc, dtype=self.dt, device=self.dev)
        V = torch.empty((kc, self.n), dtype=self.dt, device=self.dev)
        r = self.plan.factors_device(U, S, V)
        return U[:r].t(), S[:r], V[:r].t()

    def close(self):
        self.plan.close()
        self.merger.close()
