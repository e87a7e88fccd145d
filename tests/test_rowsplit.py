"""Row-band split of one matrix over ranks (paper_1710_02812_gb300.rowsplit)
on CPU: the partition, the exchange schedule and the whole driver run by
world-size 2 and 3 gloo process groups.

The ranks' computing side here is HostBand, a test double that performs each
stage with the FP64 oracle's steps on host arrays (block SVDs, MAT merges,
slab steps) and plain numpy for the CholeskyQR2 of the recovery, so the
driver's schedule (who sends what to whom, in which order, which sums and
extrema the ranks take) is exercised exactly as the GPU run uses it, and its
result can be compared with the oracle on the whole matrix."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from oracle import hmat as H
from paper_1710_02812_gb300 import rowsplit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_band_rows_cover_the_slabs_in_order():
    for m, br, world in [(1000, 100, 3), (1024, 128, 8), (1000, 128, 2), (130, 64, 3), (64, 64, 1)]:
        bands = rowsplit.band_rows(m, br, world)
        assert len(bands) == world
        assert bands[0][0] == 0 and sum(r for _, r in bands) == m
        for (a0, ar), (b0, _) in zip(bands, bands[1:]):
            assert a0 + ar == b0                   # contiguous
        for r0, rows in bands[:-1]:
            assert r0 % br == 0 and rows % br == 0  # whole slabs (the last may be ragged)
        slabs = [(rows + br - 1) // br for _, rows in bands]
        assert max(slabs) - min(slabs) <= 1         # balanced
    with pytest.raises(ValueError):
        rowsplit.band_rows(100, 64, 3)              # two slabs cannot feed three ranks


@pytest.mark.parametrize("world", [1, 2, 3, 4, 5, 7, 8, 13])
def test_merge_schedule_is_the_paper_tree_over_ranks(world):
    """Level l pairs (r, r + 2^l): the oracle's DoMergeOfSlices schedule on
    `world` elements, with element i of level l standing for rank i 2^l."""
    ours = rowsplit.merge_schedule(world)
    ref = H.tree_schedule(world)
    assert len(ours) == len(ref)
    for lv, (a, b) in enumerate(zip(ours, ref)):
        assert a == [(i << lv, j << lv) for i, j in b]
    # every rank but 0 sends exactly once, to a smaller rank
    senders = [s for lv in ours for _, s in lv]
    assert sorted(senders) == list(range(1, world))


# ---------------------------------------------------------------- the driver under gloo

class HostBand:
    """Each stage of a band with the oracle's steps in FP64 (test double)."""

    def __init__(self, x_band, n, row0, br, bc, k):
        import torch
        self.torch = torch
        self.x, self.n, self.row0, self.k = np.asarray(x_band, np.float64), n, row0, k
        self.br, self.bc = br, bc
        self.rule = H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-12)
        self.log = []

    def _pack(self, v, s):
        k, n = self.k, self.n
        pkt = np.zeros(n * k + k + 1)
        r = s.size
        pkt[:n * k].reshape(k, n)[:r] = v.T
        pkt[n * k:n * k + r] = s
        pkt[-1] = r
        return self.torch.from_numpy(pkt)

    def _unpack(self, pkt):
        p = pkt.numpy()
        k, n = self.k, self.n
        r = int(p[-1])
        return p[:n * k].reshape(k, n)[:r].T.copy(), p[n * k:n * k + r].copy(), r

    def empty_packet(self):
        return self.torch.zeros(self.n * self.k + self.k + 1, dtype=self.torch.float64)

    def local_root(self):
        rows, cols = H.grid(self.x.shape[0], self.n, self.br, self.bc)
        slabs = []
        for r0, r1 in rows:
            xj = self.x[r0:r1]
            leaves = [H.block_svd(xj[:, c0:c1], self.rule) for c0, c1 in cols]
            uj, _ = H.merge_tree(leaves, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], self.rule))
            slabs.append(H.slab_step(uj, xj, self.rule))
        v, s = H.merge_tree(slabs, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], self.rule))
        self.log.append(("root", v.shape))
        return self._pack(v, s)

    def merge(self, a, b):
        va, sa, _ = self._unpack(a)
        vb, sb, _ = self._unpack(b)
        self.log.append(("merge", va.shape, vb.shape))
        return self._pack(*H.mat_merge(va, sa, vb, sb, self.rule))

    def _pad(self, g):
        out = np.zeros((self.k, self.k))
        out[:g.shape[0], :g.shape[1]] = g
        return self.torch.from_numpy(out.reshape(-1))

    def recover_begin(self, pkt):
        self.vhat, _, self.r = self._unpack(pkt)
        self.y = self.x @ self.vhat
        return self._pad(self.y.T @ self.y)

    def recover_orth(self, gsum):
        r = self.r
        self.r1 = np.linalg.cholesky(gsum.numpy().reshape(self.k, self.k)[:r, :r]).T
        self.q = np.linalg.solve(self.r1.T, self.y.T).T
        return self._pad(self.q.T @ self.q)

    def recover_core(self, g2sum):
        r = self.r
        r2 = np.linalg.cholesky(g2sum.numpy().reshape(self.k, self.k)[:r, :r]).T
        q2 = np.linalg.solve(r2.T, self.q.T).T
        a, s, wt = np.linalg.svd(r2 @ self.r1)
        self.u, self.s, self.v = q2 @ a, s, self.vhat @ wt.T
        amax = np.zeros(self.k)
        amax[:r] = np.abs(self.u).max(axis=0) if self.u.shape[0] else 0.0
        return self.torch.from_numpy(amax)

    def recover_signs(self, amax_all):
        key = np.full(self.k, np.iinfo(np.int64).max, dtype=np.int64)
        for c in range(self.r):
            hit = np.nonzero(np.abs(self.u[:, c]) == amax_all.numpy()[c])[0]
            if hit.size:
                i = int(hit[0])
                key[c] = 2 * (self.row0 + i) + (1 if self.u[i, c] < 0 else 0)
        return self.torch.from_numpy(key)

    def recover_finish(self, key_min):
        for c, kk in enumerate(key_min.numpy()[:self.r]):
            if kk != np.iinfo(np.int64).max and kk & 1:
                self.u[:, c] *= -1
                self.v[:, c] *= -1

    def factors(self):
        return self.u, self.s, self.v


class RecordingComm:
    """TorchComm that logs every call (kind, peer or op, element count)."""

    def __init__(self):
        self.inner = rowsplit.TorchComm()
        self.rank, self.world = self.inner.rank, self.inner.world
        self.log = []

    def send(self, t, dst):
        self.log.append(["send", dst, t.numel()])
        self.inner.send(t, dst)

    def recv(self, t, src):
        self.log.append(["recv", src, t.numel()])
        self.inner.recv(t, src)

    def broadcast(self, t, src):
        self.log.append(["broadcast", src, t.numel()])
        self.inner.broadcast(t, src)

    def all_reduce(self, t, op):
        self.log.append(["all_reduce", op, t.numel()])
        self.inner.all_reduce(t, op)


RANK_CODE = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, {root!r})
    sys.path.insert(0, os.path.join({root!r}, "tests"))
    import numpy as np
    import torch.distributed as dist
    from paper_1710_02812_gb300 import rowsplit, workloads as W
    from test_rowsplit import HostBand, RecordingComm
    dist.init_process_group("gloo")
    comm = RecordingComm()
    m, n, br, bc, k = {m}, {n}, {br}, {bc}, {k}
    x = W.planted(m, n, {s!r}, noise={noise}, tag=91)
    row0, rows = rowsplit.band_rows(m, br, comm.world)[comm.rank]
    band = HostBand(x[row0:row0 + rows], n, row0, br, bc, k)
    u, s, v = rowsplit.factor_rows(band, comm)
    np.save(os.path.join({out!r}, f"u{{comm.rank}}.npy"), u)
    np.save(os.path.join({out!r}, f"s{{comm.rank}}.npy"), s)
    np.save(os.path.join({out!r}, f"v{{comm.rank}}.npy"), v)
    print(json.dumps({{"rank": comm.rank, "comm": comm.log, "band": band.log, "row0": row0, "rows": rows}}))
    dist.destroy_process_group()
""")


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _run_ranks(world, tmp_path, m, n, br, bc, k, s, noise):
    port = _free_port()
    code = RANK_CODE.format(root=ROOT, m=m, n=n, br=br, bc=bc, k=k, s=list(map(float, s)), noise=noise,
                            out=str(tmp_path))
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e[-3000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return sorted(outs, key=lambda d: d["rank"])


@pytest.mark.parametrize("world", [2, 3])
def test_driver_under_gloo_equals_the_oracle_on_the_whole_matrix(world, tmp_path):
    """4 slabs per rank (a power of two): the distributed tree is the paper's,
    so the bands' U rows, S and V equal the oracle's on the whole matrix."""
    br, bc, k = 24, 40, 6
    m, n = 4 * br * world, 200
    s = 0.7 ** np.arange(12)
    outs = _run_ranks(world, tmp_path, m, n, br, bc, k, s, 1e-7)
    from paper_1710_02812_gb300 import workloads as W
    x = W.planted(m, n, s, noise=1e-7, tag=91)
    ref = H.hmat_svd(x, br, bc, H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-12))
    u = np.concatenate([np.load(tmp_path / f"u{r}.npy") for r in range(world)])
    for r in range(world):
        np.testing.assert_allclose(np.load(tmp_path / f"s{r}.npy"), ref.s, rtol=1e-11)
        np.testing.assert_allclose(np.load(tmp_path / f"v{r}.npy"), ref.v, atol=1e-9)   # signs included
    np.testing.assert_allclose(u, ref.u, atol=1e-9)

    # the messages: the tree's sends and receives, one broadcast of V_hat,
    # two Gram sums, a maximum and a minimum over k values
    pkt = n * k + k + 1
    sched = rowsplit.merge_schedule(world)
    for d in outs:
        r = d["rank"]
        p2p = [c for c in d["comm"] if c[0] in ("send", "recv")]
        expect = []
        for lv in sched:
            for recv, send in lv:
                if r == send:
                    expect.append(["send", recv, pkt])
                elif r == recv:
                    expect.append(["recv", send, pkt])
        assert p2p == expect
        assert [c for c in d["comm"] if c[0] not in ("send", "recv")] == [
            ["broadcast", 0, pkt], ["all_reduce", "sum", k * k], ["all_reduce", "sum", k * k],
            ["all_reduce", "max", k], ["all_reduce", "min", k]]
        assert d["rows"] == 4 * br and d["row0"] == 4 * br * r
        assert sum(1 for e in d["band"] if e[0] == "merge") == sum(1 for c in p2p if c[0] == "recv")


def test_driver_under_gloo_with_ragged_bands(tmp_path):
    """Three ranks over 7 slabs (3, 2, 2) and a ragged last slab: the tree is
    local trees then the tree over ranks; the result equals the oracle's steps
    composed in that order, and the sign rule holds on the gathered U."""
    br, bc, k, world = 20, 32, 5, 3
    m, n = 7 * br - 7, 150
    s = 0.6 ** np.arange(10)
    _run_ranks(world, tmp_path, m, n, br, bc, k, s, 1e-8)
    from paper_1710_02812_gb300 import workloads as W
    x = W.planted(m, n, s, noise=1e-8, tag=91)
    rule = H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-12)
    roots = []
    for row0, rows in rowsplit.band_rows(m, br, world):
        band = x[row0:row0 + rows]
        rws, cols = H.grid(rows, n, br, bc)
        slabs = []
        for r0, r1 in rws:
            leaves = [H.block_svd(band[r0:r1, c0:c1], rule) for c0, c1 in cols]
            uj, _ = H.merge_tree(leaves, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], rule))
            slabs.append(H.slab_step(uj, band[r0:r1], rule))
        roots.append(H.merge_tree(slabs, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], rule)))
    vh, _ = H.merge_tree(roots, lambda a, b, lv, i: H.mat_merge(a[0], a[1], b[0], b[1], rule))
    uu, ss, vv = H.normalise_signs(*H.recover_left(x, vh))
    u = np.concatenate([np.load(tmp_path / f"u{r}.npy") for r in range(world)])
    np.testing.assert_allclose(np.load(tmp_path / "s0.npy"), ss, rtol=1e-11)
    np.testing.assert_allclose(u, uu, atol=1e-9)
    np.testing.assert_allclose(np.load(tmp_path / "v2.npy"), vv, atol=1e-9)
    idx = np.argmax(np.abs(u), axis=0)
    assert np.all(u[idx, np.arange(u.shape[1])] > 0)
