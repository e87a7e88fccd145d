"""The no-allocation entry point (hsvd_block_svd_noalloc).

Some callers cannot call cudaMalloc: code that runs under a memory allocator
it does not own (a framework's caching allocator, a memory-capped service),
or that must not add device allocations while other work is in flight.  For
them the library computes the rank-k SVD of one block from a fixed device
array of its own.  This file checks that entry point through the C ABI:

* against the planned path (hsvd_plan + hsvd_run on a 1 x 1 grid, the same
  block step) within the FP32 tolerance the parity tests use, and against the
  FP64 oracle's exact truncated block SVD (oracle.block_svd) on spectra where
  the randomised range finder has converged;
* on calls in a row with different shapes, so leftover contents of the shared
  array never leak into a result;
* on a rank-deficient block (rank below k: S is zero past the rank), without
  power steps, and on a block smaller than the sketch width 2k;
* its status bits on a non-finite input.

Kept in a file of its own, collected last."""
import numpy as np
import pytest
import torch

import oracle
from oracle import hmat as H
from paper_1710_02812_gb300 import hsvd
from paper_1710_02812_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIGMA_TOL = 1e-4   # FP32 path tolerance of tests/test_gpu_parity.py
ANGLE_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def planned(x, k, q):
    m, n = x.shape
    plan = hsvd.Plan(m, n, m, n, "fixed_k", k, prec="f32", power_iters=q if q > 0 else -1)
    plan.run([torch.from_numpy(x).cuda()])
    return plan.factors(0)


def noalloc(x, k, q):
    m, n = x.shape
    a = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    U = torch.full((k, m), float("nan"), dtype=torch.float32, device="cuda")  # column-major m x k
    S = torch.full((k,), float("nan"), dtype=torch.float32, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    f = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    code = hsvd.hsvd_block_svd_noalloc(a, m, n, k, q, U, S, r, flags=f)
    assert code == hsvd.HSVD_OK, hsvd.error_string(code)
    torch.cuda.synchronize()
    rank = int(r.item())
    return U[:rank].cpu().numpy().T, S[:rank].cpu().numpy(), S.cpu().numpy(), int(f.item())


# (x, k, power steps, planted spectrum, gate against the exact block SVD)
def _cases():
    s1 = np.exp(-np.arange(300) / 20.0)
    s2 = 0.93 ** np.arange(120)
    s3 = np.array([3.0, 2.0, 1.3, 0.8, 0.5])
    s4 = 0.85 ** np.arange(30)
    return [
        ("exp-decay 700x900 k=32 q=2", W.exp_decay(700, 900, r=300, noise=1e-5, tag=61, dtype=np.float32), 32, 2,
         s1),
        ("geometric 1024x640 k=48 q=1", W.planted(1024, 640, s2, noise=1e-6, tag=62).astype(np.float32), 48, 1, s2),
        ("rank 5 < k=16, q=1", W.planted(300, 260, s3, noise=0.0, tag=63).astype(np.float32), 16, 1, s3),
        ("no power steps, 512x384 k=24", W.planted(512, 384, s4, noise=0.0, tag=64).astype(np.float32), 24, 0, s4),
        ("40x30 block, sketch 30 < 2k, k=32", W.planted(40, 30, s4, noise=0.0, tag=65).astype(np.float32), 32, 1,
         s4),
    ]


def test_noalloc_matches_planned_path_and_oracle():
    for label, x, k, q, s_true in _cases():        # calls in a row, different shapes
        u_ref, s_ref, _ = planned(x, k, q)
        u, s, s_full, flags = noalloc(x, k, q)
        assert flags in (0, 2), f"{label}: status bits {flags}"   # 2: dependent directions dropped (rank < k)
        assert s.size == s_ref.size, f"{label}: rank {s.size} vs planned {s_ref.size}"
        assert np.all(s_full[s.size:] == 0), f"{label}: S past the rank {s_full[s.size:]}"
        ex_u, ex_s = H.block_svd(x.astype(np.float64), H.Rule("fixed_k", k, rank_cap=k, rank_tol=1e-5))
        assert s.size == ex_s.size, f"{label}: rank {s.size} vs exact {ex_s.size}"
        j = oracle.gap_prefix(s_true, s.size)
        assert j > 0
        for ref_u, ref_s, what in ((u_ref, s_ref, "planned path"), (ex_u, ex_s, "oracle block SVD")):
            err = oracle.sigma_rel_err(s, ref_s, j)
            assert err <= SIGMA_TOL, f"{label}: sigma rel err {err:.3e} against the {what}"
            ang = oracle.leading_subspace_angle(u, ref_u, ref_s, upto=j)
            assert ang <= ANGLE_TOL, f"{label}: angle {ang:.3e} against the {what}"
        assert oracle.orthonormality_defect(u) < 1e-4


def test_noalloc_reports_nonfinite_input():
    x = W.planted(200, 160, 0.8 ** np.arange(20), noise=1e-6, tag=66).astype(np.float32)
    x[17, 33] = np.nan
    _, _, _, flags = noalloc(x, 8, 1)
    assert flags & 4, f"status bits {flags}"
    x[17, 33] = 0.5                                 # the next clean call reports clean again
    _, s, _, flags = noalloc(x, 8, 1)
    assert flags == 0 and s.size == 8 and np.all(np.isfinite(s))


def test_noalloc_rejects_sizes_beyond_the_limit():
    a = torch.zeros((8, 2048), dtype=torch.float32, device="cuda")
    U = torch.zeros((65, 8), dtype=torch.float32, device="cuda")
    S = torch.zeros(65, dtype=torch.float32, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert hsvd.hsvd_block_svd_noalloc(a, 8, 2048, 4, 1, U, S, r) == hsvd.HSVD_EUNSUPPORTED
    a16 = a[:, :16]
    assert hsvd.hsvd_block_svd_noalloc(a16, 8, 16, 65, 1, U, S, r) == hsvd.HSVD_EUNSUPPORTED
    assert hsvd.hsvd_block_svd_noalloc(a16, 8, 16, 0, 1, U, S, r) == hsvd.HSVD_EINVAL
