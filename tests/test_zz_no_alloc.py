"""The no-allocation entry point (hsvd_block_svd_noalloc) against the planned
path: callers that cannot allocate device memory get the rank-k SVD of one
block from a fixed device array inside the library, and it must agree with
hsvd_plan + hsvd_run on a 1 x 1 grid (the same block step) within the FP32
tolerance the parity tests use.  Two calls in a row on different matrices
check that the shared array's leftover contents never leak into a result.

Kept in a file of its own, collected last."""
import numpy as np
import pytest
import torch

import oracle
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
    plan = hsvd.Plan(m, n, m, n, "fixed_k", k, prec="f32", power_iters=q)
    plan.run([torch.from_numpy(x).cuda()])
    return plan.factors(0)


def noalloc(x, k, q):
    m, n = x.shape
    a = torch.from_numpy(x).cuda()
    U = torch.full((k, m), float("nan"), dtype=torch.float32, device="cuda")  # column-major m x k
    S = torch.full((k,), float("nan"), dtype=torch.float32, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = hsvd.hsvd_block_svd_noalloc(a, m, n, k, q, U, S, r)
    assert code == hsvd.HSVD_OK, hsvd.error_string(code)
    torch.cuda.synchronize()
    rank = int(r.item())
    return U[:rank].cpu().numpy().T, S[:rank].cpu().numpy(), S.cpu().numpy()


def test_noalloc_matches_planned_path_twice():
    cases = [
        (W.exp_decay(700, 900, r=300, noise=1e-5, tag=61, dtype=np.float32), 32, 2, np.exp(-np.arange(300) / 20.0)),
        (W.planted(1024, 640, 0.93 ** np.arange(120), noise=1e-6, tag=62).astype(np.float32), 48, 1,
         0.93 ** np.arange(120)),
    ]
    for x, k, q, s_true in cases:          # two calls in a row, different shapes
        u_ref, s_ref, _ = planned(x, k, q)
        u, s, s_full = noalloc(x, k, q)
        assert s.size == s_ref.size == k
        assert np.all(s_full[s.size:] == 0)
        j = oracle.gap_prefix(s_true, k)
        assert j > 0
        err = oracle.sigma_rel_err(s, s_ref, j)
        assert err <= SIGMA_TOL, f"sigma rel err {err:.3e}"
        ang = oracle.leading_subspace_angle(u, u_ref, s_ref, upto=j)
        assert ang <= ANGLE_TOL, f"angle {ang:.3e}"
        assert oracle.orthonormality_defect(u) < 1e-4


def test_noalloc_rejects_sizes_beyond_the_limit():
    a = torch.zeros((8, 2048), dtype=torch.float32, device="cuda")
    U = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    S = torch.zeros(4, dtype=torch.float32, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert hsvd.hsvd_block_svd_noalloc(a, 8, 2048, 4, 1, U, S, r) == hsvd.HSVD_EUNSUPPORTED
    assert hsvd.hsvd_block_svd_noalloc(a, 8, 16, 65, 1, U, S, r) == hsvd.HSVD_EUNSUPPORTED
    assert hsvd.hsvd_block_svd_noalloc(a, 8, 16, 0, 1, U, S, r) == hsvd.HSVD_EINVAL
