"""The row-band split (paper_1710_02812_gb300.rowsplit) on the GPU, through
the C ABI: band plans stopped after their row trees, merge plans for the tree
over ranks, and the staged recovery of U with the sums over bands.

This run has one GPU, so the ranks are emulated by host threads of one
process, each driving its own band plan on the same device; their exchanges
(ThreadComm) are host-side copies and reductions between kernel launches.
No kernel of one rank waits on another rank.  The distributed result is
compared with the single-plan path on the whole matrix and with the oracle
(the same tree: a power of two of slabs per rank)."""
from __future__ import annotations

import queue
import threading

import numpy as np
import pytest
import torch

import oracle
from oracle import hmat as H
from paper_1710_02812_gb300 import hsvd, rowsplit
from paper_1710_02812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


class ThreadComm:
    """factor_rows' communicator for ranks emulated by threads of one process."""

    def __init__(self, shared, rank):
        self.s, self.rank, self.world = shared, rank, shared["world"]

    def _sync(self):
        torch.cuda.synchronize()

    def send(self, t, dst):
        self._sync()
        self.s["q"][(self.rank, dst)].put(t.clone())

    def recv(self, t, src):
        t.copy_(self.s["q"][(src, self.rank)].get(timeout=120))
        self._sync()

    def broadcast(self, t, src):
        self._sync()
        if self.rank == src:
            self.s["slot"][src] = t.clone()
        self.s["bar"].wait(timeout=120)
        if self.rank != src:
            t.copy_(self.s["slot"][src])
        self._sync()
        self.s["bar"].wait(timeout=120)

    def all_reduce(self, t, op):
        self._sync()
        self.s["slot"][self.rank] = t.clone()
        self.s["bar"].wait(timeout=120)
        acc = self.s["slot"][0].clone()
        for r in range(1, self.world):
            v = self.s["slot"][r]
            acc = acc + v if op == "sum" else (torch.maximum(acc, v) if op == "max" else torch.minimum(acc, v))
        t.copy_(acc)
        self._sync()
        self.s["bar"].wait(timeout=120)


def run_split(x, world, br, bc, k, prec, **kw):
    """Factor x with `world` emulated ranks; returns gathered (U, S, V) on the host."""
    m, n = x.shape
    xd = torch.from_numpy(x).cuda()
    shared = {"world": world, "bar": threading.Barrier(world), "slot": [None] * world,
              "q": {(a, b): queue.Queue() for a in range(world) for b in range(world)}}
    results, errors = [None] * world, []
    bands = rowsplit.band_rows(m, br, world)
    first_run = threading.Lock()

    def rank_main(r):
        try:
            row0, rows = bands[r]
            # a plan's first run captures its CUDA graph: plans are made and
            # first run one thread at a time, and every thread waits for all of
            # them before the split (a device-wide synchronise of one thread
            # may not overlap another's capture)
            with first_run:
                band = rowsplit.DeviceBand(xd[row0:row0 + rows], n, row0, br, bc, k, prec=prec, **kw)
                band.plan.run([band.x])
                torch.cuda.synchronize()
            shared["bar"].wait(timeout=300)
            u, s, v = rowsplit.factor_rows(band, ThreadComm(shared, r))
            results[r] = (u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy(), band.plan.status())
            band.close()
        except Exception as e:  # reported by the main thread
            errors.append((r, repr(e)))
            shared["bar"].abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errors, errors
    u = np.concatenate([results[r][0] for r in range(world)])
    for r in range(1, world):
        np.testing.assert_array_equal(results[r][1], results[0][1])   # every rank holds the same S and V
        np.testing.assert_array_equal(results[r][2], results[0][2])
    return u, results[0][1], results[0][2], [results[r][3] for r in range(world)]


@pytest.mark.parametrize("world", [2, 4])
def test_fp64_split_equals_the_oracle(world):
    br, bc, k = 128, 160, 12
    m, n = 2 * br * world, 700
    s_true = 0.8 ** np.arange(60)
    x = W.planted(m, n, s_true, noise=1e-9, tag=301 + world)
    u, s, v, sts = run_split(x, world, br, bc, k, "f64")
    ref = H.hmat_svd(x, br, bc, H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-12))
    assert s.size == ref.s.size == k
    assert oracle.sigma_rel_err(s, ref.s, k) <= 1e-10
    # vectors with their signs (the sign rule agreed over the bands)
    np.testing.assert_allclose(u, ref.u, rtol=0, atol=1e-6)
    np.testing.assert_allclose(v, ref.v, rtol=0, atol=1e-6)
    assert all(st["nonfinite"] == 0 and st["not_converged"] == 0 for st in sts)


@pytest.mark.parametrize("prec", ["f32", "bf16_mixed"])
def test_split_equals_the_single_plan(prec):
    """Three ranks over 8 slabs (3, 3, 2): the split result against hsvd_run
    on the whole matrix with the same tree order only where they coincide, so
    compared at the FP32 tolerance on the leading gap-separated modes, and
    against the oracle composed in the split's order."""
    br, bc, k, world = 256, 256, 16, 3
    m, n = 8 * br, 1536
    # a gap after mode k: the truncations are nearly lossless, so the two tree
    # orders agree far below the tolerance
    s_true = np.concatenate([np.exp(-np.arange(k) / 8.0), 1e-3 * np.exp(-np.arange(k, 200) / 8.0)])
    x = W.planted(m, n, s_true, noise=1e-6, tag=311).astype(np.float32)
    xin = W.bf16_round(x) if prec == "bf16_mixed" else x
    u, s, v, sts = run_split(x, world, br, bc, k, prec, power_iters=2)
    # the oracle in the split's order: local trees, then the tree over ranks
    rule = H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-5)
    xd = xin.astype(np.float64)
    roots = []
    for row0, rows in rowsplit.band_rows(m, br, world):
        rws, cols = H.grid(rows, n, br, bc)
        slabs = []
        for r0, r1 in rws:
            xj = xd[row0 + r0:row0 + r1]
            leaves = [H.block_svd(xj[:, c0:c1], rule) for c0, c1 in cols]
            uj, _ = H.merge_tree(leaves, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], rule))
            slabs.append(H.slab_step(uj, xj, rule))
        roots.append(H.merge_tree(slabs, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], rule)))
    vh, _ = H.merge_tree(roots, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], rule))
    ru, rs, rv = H.normalise_signs(*H.recover_left(xd, vh))
    j = oracle.gap_prefix(s_true, k)
    assert s.size == k and j > 0
    assert oracle.sigma_rel_err(s, rs, j) <= 1e-4
    assert oracle.leading_subspace_angle(u, ru, rs, upto=j) <= 1e-3
    assert oracle.leading_subspace_angle(v, rv, rs, upto=j) <= 1e-3
    idx = np.argmax(np.abs(u), axis=0)
    assert np.all(u[idx, np.arange(u.shape[1])] > 0)
    assert all(st["nonfinite"] == 0 and st["tensor_timeouts"] == 0 for st in sts)
    # and the single-plan path on the whole matrix (the paper's tree)
    plan = hsvd.Plan(m, n, br, bc, "fixed_k", k, prec=prec, power_iters=2)
    plan.run([torch.from_numpy(x).cuda()])
    pu, ps, pv = plan.factors(0)
    assert oracle.sigma_rel_err(s, ps, j) <= 1e-4


def test_merge_plan_against_the_oracle_merge():
    """hsvd_merge_run: the MAT merge of two factor pairs (Section 3) against
    the oracle's plain concatenated-SVD merge, FP64."""
    h, k = 900, 10
    g = np.random.default_rng(5)
    u1, _ = np.linalg.qr(g.standard_normal((h, k)))
    u2, _ = np.linalg.qr(g.standard_normal((h, k)))
    u2[:, :4] = u1[:, :4] + 1e-3 * g.standard_normal((h, 4))          # overlapping subspaces
    u2, _ = np.linalg.qr(u2)
    s1, s2 = np.linspace(5, 1, k), np.linspace(4, 0.5, k)
    mp = hsvd.MergePlan(h, "fixed_k", k, prec="f64")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mp.run(dev(u1.T), dev(s1), k, dev(u2.T), dev(s2), k)
    V = torch.empty((k, h), dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    r = mp.root(V, S)
    ru, rs = H.mat_merge(u1, s1, u2, s2, H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-12))
    assert r == k
    np.testing.assert_allclose(S.cpu().numpy(), rs, rtol=1e-11)
    assert oracle.principal_angle(V.cpu().numpy()[:r].T, ru) < 1e-9
    # a rank below the cap: the factors past it are ignored
    mp.run(dev(u1.T), dev(s1), 6, dev(u2.T), dev(s2), 3)
    r = mp.root(V, S)
    ru, rs = H.mat_merge(u1[:, :6], s1[:6], u2[:, :3], s2[:3], H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-12))
    assert r == rs.size == 9
    np.testing.assert_allclose(S.cpu().numpy()[:r], rs, rtol=1e-11)
    assert np.all(S.cpu().numpy()[r:] == 0)
