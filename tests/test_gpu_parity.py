"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated per precision):
  * FP64 path: top-k sigma relative error <= 1e-10; subspace angle over
    gap-separated leading groups <= 1e-6 rad.
  * FP32 and BF16-mixed paths: top-k sigma relative error <= 1e-4; subspace
    angle <= 1e-3 rad.
  * Every path: Frobenius reconstruction error ||X - U S V^T|| / ||X|| within
    1% of the oracle's, plus a rounding floor of 50 u of the path (an exactly
    low-rank input makes the oracle's own error a rounding residue).
The oracle consumes the same bytes as the GPU (BF16 inputs are rounded
first), and uses the same rank tolerance, so rank decisions agree.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import hmat as H
from paper_1710_02812_gb300 import hsvd
from paper_1710_02812_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT_REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

TOL = {"f64": (1e-10, 1e-6, 1.1e-16), "f32": (1e-4, 1e-3, 6e-8), "bf16_mixed": (1e-4, 1e-3, 6e-8)}
RANK_TOL = {"f64": 1e-12, "f32": 1e-5, "bf16_mixed": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def to_device(x, prec):
    if prec == "f64":
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def run_gpu(xs, br, bc, mode, param, prec, rank_cap=None, tree="col_then_row", **kw):
    m = [x.shape[0] for x in xs]
    n = [x.shape[1] for x in xs]
    plan = hsvd.Plan(m, n, br, bc, mode, param, rank_cap=rank_cap, tree=tree, prec=prec, **kw)
    dev = [to_device(x, prec) for x in xs]
    plan.run(dev)
    torch.cuda.synchronize()
    outs = [plan.factors(i) for i in range(len(xs))]
    st = plan.status()
    return outs, st, plan


def recon(x, u, s, v):
    xd = np.asarray(x, dtype=np.float64)
    nx = np.linalg.norm(xd)
    return float(np.linalg.norm(xd - (u.astype(np.float64) * s) @ v.T.astype(np.float64)) / nx) if nx else 0.0


def check(x, got, ref, prec, label, s_true, recon_ulps=50):
    """Gate sigma and subspaces on the leading gap-separated prefix of the
    planted spectrum s_true (values inside a dense cluster, e.g. a noise bulk, are not
    determined to the tolerance); the rest is checked loosely, normwise.  The
    reconstruction error must be within 1% of the oracle's plus recon_ulps
    units of the path's rounding."""
    u, s, v = got
    stol, atol, eps = TOL[prec]
    assert s.size == ref.s.size, f"{label}: rank {s.size} vs oracle {ref.s.size}"
    if s.size == 0:
        return
    j = oracle.gap_prefix(s_true, s.size)
    assert j > 0, f"{label}: no gap-separated prefix"
    err = oracle.sigma_rel_err(s, ref.s, j)
    assert err <= stol, f"{label}: sigma rel err {err:.3e} > {stol} over the first {j}"
    au = oracle.leading_subspace_angle(u, ref.u, ref.s, upto=j)
    av = oracle.leading_subspace_angle(v, ref.v, ref.s, upto=j)
    assert au <= atol and av <= atol, f"{label}: angles U {au:.3e} V {av:.3e} > {atol}"
    normwise = float(np.max(np.abs(s - ref.s)) / ref.s[0])
    assert normwise <= max(1e-2, stol), f"{label}: normwise sigma err {normwise:.3e}"
    rg, ro = recon(x, u, s, v), recon(x, ref.u, ref.s, ref.v)
    assert abs(rg - ro) <= 0.01 * ro + recon_ulps * eps, f"{label}: recon {rg:.6e} vs oracle {ro:.6e}"
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)


def oracle_run(x, br, bc, mode, param, prec, rank_cap=256, tree="col_then_row"):
    rule = H.Rule(mode, param, rank_cap=rank_cap, rank_tol=RANK_TOL[prec])
    return H.hmat_svd(np.asarray(x, dtype=np.float64), br, bc, rule, tree=tree)


# ---------------------------------------------------------------- FP64

def test_fp64_fixed_rank_512_parity():
    """The 512 x 512, rank-10 + 1e-6 noise, 4 x 4 grid of 128^2, k = 10 case."""
    x, cfg = W.fixed_rank_512()
    (got,), st, _ = run_gpu([x], 128, 128, "fixed_k", 10, "f64")
    ref = oracle_run(x, 128, 128, "fixed_k", 10, "f64")
    check(x, got, ref, "f64", "fixed_rank_512", s_true=10.0 ** (-np.arange(10) / 3.0))
    assert st["not_converged"] == 0 and st["nonfinite"] == 0


@pytest.mark.parametrize("m,n,br,bc,k", [
    (700, 900, 256, 192, 12),   # ragged slabs and slices, 3 x 5 grid
    (300, 200, 300, 200, 8),    # 1 x 1 grid: truncated SVD of the whole matrix
    (520, 130, 40, 130, 6),     # 13 x 1 grid: row tree only, odd leaf count
    (96, 1000, 96, 70, 6),      # 1 x 15 grid: column tree only
    (257, 263, 64, 64, 20),     # ragged tail of 1-2 rows/cols, k' capped by block
])
def test_fp64_grids(m, n, br, bc, k):
    s = 0.8 ** np.arange(min(m, n, 60))
    x = W.planted(m, n, s, noise=1e-9, tag=m + 7 * n)
    (got,), st, _ = run_gpu([x], br, bc, "fixed_k", k, "f64")
    ref = oracle_run(x, br, bc, "fixed_k", k, "f64")
    check(x, got, ref, "f64", f"{m}x{n}/{br}x{bc}", s_true=s)


def test_fp64_exact_rank_recovery():
    s = np.array([4.0, 2.5, 1.0, 0.4])
    x, u0, s0, v0 = W.planted(333, 444, s, noise=0.0, tag=9, return_factors=True)
    (got,), st, _ = run_gpu([x], 100, 120, "fixed_k", 8, "f64")
    u, sg, v = got
    assert sg.size == 4
    np.testing.assert_allclose(sg, s, rtol=1e-10)
    assert oracle.principal_angle(u, u0) < 1e-8 and oracle.principal_angle(v, v0) < 1e-8


def test_fp64_row_then_col():
    x, _ = W.fixed_rank_512()
    x = x[:400, :300]
    (got,), _, _ = run_gpu([x], 96, 128, "fixed_k", 10, "f64", tree="row_then_col")
    ref = oracle_run(x, 96, 128, "fixed_k", 10, "f64", tree="row_then_col")
    check(x, got, ref, "f64", "row_then_col", s_true=np.linalg.svd(x, compute_uv=False)[:10])


def _largest_entry_positive(u):
    """The output sign rule: the largest-magnitude entry of each U column is
    positive."""
    idx = np.argmax(np.abs(u), axis=0)
    return bool(np.all(u[idx, np.arange(u.shape[1])] > 0))


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16_mixed"])
@pytest.mark.parametrize("tree", ["col_then_row", "row_then_col"])
def test_signs_match_oracle_elementwise(prec, tree):
    """U and V compared entry by entry WITH their signs (no abs, no angles): on
    an exactly rank-6 input with well separated values every singular vector
    is unique up to sign, so the device's sign normalisation must give the
    oracle's vectors themselves.  The rule (largest-magnitude entry of each U
    column positive) is also checked on the device output directly."""
    s = np.array([4.0, 2.5, 1.6, 1.0, 0.6, 0.35])
    x = W.planted(296, 264, s, noise=0.0, tag=31)
    xin = W.bf16_round(x) if prec == "bf16_mixed" else x
    (got,), st, _ = run_gpu([xin], 80, 72, "fixed_k", 6, prec, tree=tree)
    u, sg, v = got
    ref = oracle_run(xin, 80, 72, "fixed_k", 6, prec, tree=tree)
    assert sg.size == ref.s.size == 6
    assert _largest_entry_positive(u)
    tol = 1e-10 if prec == "f64" else 1e-3
    np.testing.assert_allclose(u, ref.u, rtol=0, atol=tol)
    np.testing.assert_allclose(v, ref.v, rtol=0, atol=tol)


# ---------------------------------------------------------------- FP32

@pytest.mark.parametrize("m,n,br,bc,k", [
    (1500, 1300, 384, 320, 32),
    (1024, 1024, 256, 256, 48),
    (777, 2049, 200, 512, 24),
])
def test_fp32_exp_decay(m, n, br, bc, k):
    x = W.exp_decay(m, n, r=min(m, n, 400), noise=1e-5, tag=m + n, dtype=np.float32)
    (got,), st, _ = run_gpu([x], br, bc, "fixed_k", k, "f32")
    ref = oracle_run(x, br, bc, "fixed_k", k, "f32")
    check(x, got, ref, "f32", f"{m}x{n}", s_true=np.exp(-np.arange(min(m, n, 400)) / 20.0))
    assert st["not_converged"] == 0 and st["nonfinite"] == 0


def test_fp32_exact_rank_recovery():
    s = np.array([3.0, 2.0, 1.5, 0.7, 0.3])
    x, u0, s0, v0 = W.planted(600, 500, s, noise=0.0, tag=12, return_factors=True)
    x = x.astype(np.float32)
    (got,), st, _ = run_gpu([x], 128, 128, "fixed_k", 16, "f32")
    u, sg, v = got
    assert sg.size == 5
    np.testing.assert_allclose(sg, s, rtol=1e-5)
    assert oracle.principal_angle(u, u0) < 1e-4 and oracle.principal_angle(v, v0) < 1e-4


def test_fp32_batch_of_uneven_matrices():
    sizes = [(600, 450, 9), (1030, 700, 20), (300, 1200, 14), (129, 131, 5)]
    xs = [W.ragged_matrix(m, n, r, tag=i) for i, (m, n, r) in enumerate(sizes)]
    # the planted tails sit within 2x of the block noise level: more power steps
    outs, st, _ = run_gpu(xs, 256, 256, "fixed_k", 24, "f32", power_iters=4)
    for (m, n, r), x, got in zip(sizes, xs, outs):
        ref = oracle_run(x, 256, 256, "fixed_k", 24, "f32")
        # k = 24 exceeds every planted rank: only the planted part is gated
        check(x, got, ref, "f32", f"batch {x.shape}", s_true=np.exp(-np.arange(r) / r) / r)


def test_fp32_gamma_mode():
    s = np.array([10.0, 7.0, 5.0, 3.0, 1.0, 0.5, 0.2, 0.05])
    x = W.planted(800, 640, s, noise=1e-6, tag=21).astype(np.float32)
    (got,), _, _ = run_gpu([x], 200, 160, "gamma", 0.02, "f32", rank_cap=32)
    ref = oracle_run(x, 200, 160, "gamma", 0.02, "f32", rank_cap=32)
    check(x, got, ref, "f32", "gamma", s_true=s)


def test_fp32_energy_mode():
    s = np.sqrt(np.array([50.0, 25.0, 12.0, 6.0, 3.0, 1.5, 0.8]))
    x = W.planted(900, 700, s, noise=1e-7, tag=22).astype(np.float32)
    (got,), _, _ = run_gpu([x], 300, 350, "energy", 0.97, "f32", rank_cap=16)
    ref = oracle_run(x, 300, 350, "energy", 0.97, "f32", rank_cap=16)
    check(x, got, ref, "f32", "energy", s_true=s)


def test_fp32_zero_matrix_and_tiny_shapes():
    (got,), st, _ = run_gpu([np.zeros((100, 80), np.float32)], 32, 32, "fixed_k", 4, "f32")
    assert got[1].size == 0
    x = np.array([[3.0]], dtype=np.float32)
    (got,), _, _ = run_gpu([x], 1, 1, "fixed_k", 1, "f32")
    np.testing.assert_allclose(got[1], [3.0], rtol=1e-6)
    x = W.planted(3, 5, [2.0, 1.0], tag=4).astype(np.float32)
    (got,), _, _ = run_gpu([x], 2, 2, "fixed_k", 2, "f32")
    ref = oracle_run(x, 2, 2, "fixed_k", 2, "f32")
    check(x, got, ref, "f32", "3x5", s_true=[2.0, 1.0])


# ---------------------------------------------------------------- mixed

def test_bf16_mixed_matches_oracle_on_rounded_input():
    x32 = W.exp_decay(1024, 1536, r=300, noise=1e-5, tag=31, dtype=np.float32)
    xb = W.bf16_round(x32)
    (got,), st, _ = run_gpu([xb], 256, 256, "fixed_k", 32, "bf16_mixed")
    ref = oracle_run(xb, 256, 256, "fixed_k", 32, "bf16_mixed")
    check(xb, got, ref, "bf16_mixed", "bf16", s_true=np.exp(-np.arange(300) / 20.0))


# ---------------------------------------------------------------- API paths

def test_run_host_equals_run_device():
    x = W.exp_decay(900, 700, r=200, noise=1e-5, tag=41, dtype=np.float32)
    plan = hsvd.Plan(900, 700, 256, 256, "fixed_k", 16, prec="f32", host_staging=True)
    plan.run([to_device(x, "f32")])
    u1, s1, v1 = plan.factors(0)
    plan.run_host([x])
    torch.cuda.synchronize()
    u2, s2, v2 = plan.factors(0)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(u1, u2)
    np.testing.assert_array_equal(v1, v2)


def test_factors_device_matches_host():
    x = W.exp_decay(500, 400, r=100, noise=1e-5, tag=42, dtype=np.float32)
    plan = hsvd.Plan(500, 400, 128, 128, "fixed_k", 8, prec="f32")
    plan.run([to_device(x, "f32")])
    u, s, v = plan.factors(0)
    U = torch.zeros((8, 500), dtype=torch.float32, device="cuda")
    V = torch.zeros((8, 400), dtype=torch.float32, device="cuda")
    S = torch.zeros(8, dtype=torch.float32, device="cuda")
    r = plan.factors_device(U, S, V, 0)
    torch.cuda.synchronize()
    assert r == s.size
    np.testing.assert_array_equal(U[:r].cpu().numpy().T, u)
    np.testing.assert_array_equal(V[:r].cpu().numpy().T, v)
    np.testing.assert_array_equal(S[:r].cpu().numpy(), s)


def test_repeat_runs_are_deterministic():
    x = W.exp_decay(700, 600, r=150, noise=1e-5, tag=43, dtype=np.float32)
    plan = hsvd.Plan(700, 600, 160, 160, "fixed_k", 12, prec="f32")
    xd = to_device(x, "f32")
    plan.run([xd])
    a = plan.factors(0)
    plan.run([xd])
    b = plan.factors(0)
    for p, q in zip(a, b):
        np.testing.assert_array_equal(p, q)


# ---------------------------------------------------------------- status words

def test_sweep_cap_reports_not_converged_without_failing():
    x = W.exp_decay(512, 512, r=200, noise=1e-5, tag=44, dtype=np.float32)
    (_,), st, _ = run_gpu([x], 128, 128, "fixed_k", 16, "f32", max_sweeps=1)
    assert st["not_converged"] > 0


def test_nonfinite_input_is_reported():
    x = W.exp_decay(256, 256, r=64, noise=1e-5, tag=45, dtype=np.float32)
    x[17, 33] = np.nan
    (_,), st, _ = run_gpu([x], 64, 64, "fixed_k", 8, "f32")
    assert st["nonfinite"] > 0


# ---------------------------------------------------------------- mixed, tensor cores

@pytest.mark.parametrize("m,n,br,bc,k", [
    (700, 900, 256, 192, 24),    # ragged 128-row tiles and K tails through the tcgen05 path
    (2048, 1536, 512, 512, 64),  # full 128-wide sketch
])
def test_bf16_mixed_tensor_core_ragged(m, n, br, bc, k):
    r = min(m, n, 300)
    xb = W.bf16_round(W.exp_decay(m, n, r=r, noise=1e-5, tag=m + 3 * n, dtype=np.float32))
    (got,), st, _ = run_gpu([xb], br, bc, "fixed_k", k, "bf16_mixed")
    assert st["tensor_timeouts"] == 0
    ref = oracle_run(xb, br, bc, "fixed_k", k, "bf16_mixed")
    check(xb, got, ref, "bf16_mixed", f"tc {m}x{n}", s_true=np.exp(-np.arange(r) / 20.0))


@pytest.mark.parametrize("m,n,br,bc,k,r,tree", [
    (700, 900, 256, 192, 56, 37, "col_then_row"),  # ranks 37 < cap 56: extents and the [U1 U_o] split set on the device
    (640, 1000, 128, 248, 64, 45, "row_then_col"),  # V-side merges, long TN products split over K
])
def test_bf16_mixed_factor_products_with_device_ranks(m, n, br, bc, k, r, tree):
    """The mixed path's factor products (merge P, Q, their CholeskyQR, U =
    [U1 U_o] U_E, slab and recovery products: the FP32-grade tensor-core
    kernels) with extents chosen on the device below their static caps: the
    input A B^T with A, B of entries in {-1, 0, 1} is exactly rank r and
    exact in BF16 (integer entries of magnitude <= r), so every block and
    merge has rank r < k (k > 32: the tensor-core kernels, not the skinny
    ones), and the second-segment offset r is not a multiple of 4; ragged
    block grids, both tree orders; compared with the oracle on the same
    values (spectrum gate from an FP64 SVD of the input)."""
    g = np.random.default_rng(8000 + r)
    a = g.integers(-1, 2, size=(m, r)).astype(np.float64)
    b = g.integers(-1, 2, size=(n, r)).astype(np.float64)
    x = (a @ b.T).astype(np.float32)
    assert np.array_equal(W.bf16_round(x), x)
    s_true = np.linalg.svd(x.astype(np.float64), compute_uv=False)[:r]
    (got,), st, _ = run_gpu([x], br, bc, "fixed_k", k, "bf16_mixed", tree=tree, power_iters=2, oversample=k)
    assert st["nonfinite"] == 0 and st["tensor_timeouts"] == 0
    ref = oracle_run(x, br, bc, "fixed_k", k, "bf16_mixed", tree=tree)
    assert ref.s.size == r
    # the oracle's residual on an exactly rank-r input is FP64 rounding, so the
    # reconstruction bound is the FP32-grade path's own: 5.6e-6 and 7.4e-6 on
    # these two inputs, the same with the SIMT products and on the plain FP32
    # path (factors orthonormal to ~4e-6); gated at 250 units of 2^-24
    check(x, got, ref, "bf16_mixed", f"device ranks {m}x{n}/{br}x{bc} k={k} r={r} {tree}", s_true=s_true,
          recon_ulps=250)


def test_bf16_mixed_factor_products_energy_batch():
    """Energy rule on a batch of two uneven matrices through the mixed path
    with a rank cap of 64: per-matrix ranks decided on the device feed the
    tensor-core factor products of both trees in one launch per level."""
    g = np.random.default_rng(77)
    xs, tops = [], []
    for j, (m, n) in enumerate([(620, 840), (900, 560)]):
        r1 = 36 + 2 * j  # slow decay: every kept value far above the energy cut, block by block
        top = np.sort(g.uniform(0.5, 2.0, r1))[::-1] * (0.97 ** np.arange(r1))
        s_true = np.concatenate([top, 1e-3 * top[-1] * 0.5 ** np.arange(6)])
        xs.append(W.bf16_round(W.planted(m, n, s_true, noise=1e-6, tag=7100 + j).astype(np.float32)))
        tops.append(top)
    outs, st, _ = run_gpu(xs, 200, 216, "energy", 0.99999, "bf16_mixed", rank_cap=64, power_iters=2, oversample=64)
    assert st["nonfinite"] == 0 and st["tensor_timeouts"] == 0
    for x, got, top in zip(xs, outs, tops):
        ref = oracle_run(x, 200, 216, "energy", 0.99999, "bf16_mixed", rank_cap=64)
        check(x, got, ref, "bf16_mixed", f"energy batch {x.shape}", s_true=top[top >= 0.05 * top[0]])


def test_bf16_mixed_bf16_input_dtype():
    """BF16 storage given directly (in_dtype bf16) reads the same values."""
    xb = W.bf16_round(W.exp_decay(768, 640, r=200, noise=1e-5, tag=71, dtype=np.float32))
    # an exp(-i/20) spectrum needs ~48 extra sketch columns for a 0.1 gap at k
    plan = hsvd.Plan(768, 640, 128, 128, "fixed_k", 16, prec="bf16_mixed", in_dtype="bf16", oversample=48)
    t = torch.from_numpy(xb).cuda().to(torch.bfloat16)
    plan.run([t])
    got = plan.factors(0)
    ref = oracle_run(xb, 128, 128, "fixed_k", 16, "bf16_mixed")
    check(xb, got, ref, "bf16_mixed", "bf16 input", s_true=np.exp(-np.arange(200) / 20.0))


def test_bf16_mixed_simt_fallback_for_unaligned_blocks():
    """Block origins off 8-element boundaries cannot be TMA tile origins:
    the mixed path then runs its products on the SIMT kernels."""
    xb = W.bf16_round(W.exp_decay(600, 500, r=150, noise=1e-5, tag=72, dtype=np.float32))
    (got,), st, _ = run_gpu([xb], 250, 190, "fixed_k", 16, "bf16_mixed", oversample=48)
    ref = oracle_run(xb, 250, 190, "fixed_k", 16, "bf16_mixed")
    check(xb, got, ref, "bf16_mixed", "simt fallback", s_true=np.exp(-np.arange(150) / 20.0))


def test_bf16_mixed_row_then_col_tensor_core():
    xb = W.bf16_round(W.exp_decay(640, 1024, r=200, noise=1e-5, tag=73, dtype=np.float32))
    (got,), st, _ = run_gpu([xb], 128, 256, "fixed_k", 20, "bf16_mixed", tree="row_then_col", oversample=48)
    ref = oracle_run(xb, 128, 256, "fixed_k", 20, "bf16_mixed", tree="row_then_col")
    check(xb, got, ref, "bf16_mixed", "tc row_then_col", s_true=np.exp(-np.arange(200) / 20.0))


# ---------------------------------------------------------------- cores on thread-block clusters

@pytest.mark.parametrize("m,n,br,bc,k", [
    (2048, 2048, 1024, 1024, 128),  # 256 x 256 block and merge cores, 8-CTA clusters
    (2048, 2048, 256, 256, 100),    # 200-row cores: 64 block cores on 2-CTA clusters, merges on 4
])
def test_fp32_wide_cores_on_clusters(m, n, br, bc, k):
    """Cores too large for one CTA (k = 128 gives 256 x 256 block sketch and
    merge cores) and levels with few cores run spread over a cluster.  The
    spectrum exp(-i/40) keeps absolute gaps near sigma_k well above FP32
    rounding of the input (a 1/i spectrum does not: an input perturbation of
    FP32 size alone turns its 99th vector by ~1e-3 rad)."""
    s_true = np.exp(-np.arange(160) / 40.0)
    x = W.planted(m, n, s_true, noise=1e-6, tag=81 + br).astype(np.float32)
    (got,), st, _ = run_gpu([x], br, bc, "fixed_k", k, "f32", power_iters=2)
    assert st["not_converged"] == 0 and st["nonfinite"] == 0
    ref = oracle_run(x, br, bc, "fixed_k", k, "f32")
    check(x, got, ref, "f32", f"clusters {m}x{n}/{br}", s_true=s_true)


# ---------------------------------------------------------------- Alg. 2 (iterative improvement)

@pytest.mark.parametrize("prec", ["f64", "f32", "bf16_mixed"])
def test_refine_matches_oracle_alg2(prec):
    """hsvd_refine runs the passes of Alg. 2 on the last run's factors; after
    the same number of passes it matches the oracle's Alg. 2 started from
    the oracle's own MAT result (both contract toward the truncated SVD)."""
    k = 12
    s_true = np.concatenate([np.linspace(4.0, 2.0, k), 0.8 * 0.9 ** np.arange(40)])
    x = W.planted(700, 520, s_true, noise=1e-6, tag=101)
    if prec == "bf16_mixed":
        x = W.bf16_round(x.astype(np.float32))
    xin = x if prec == "f64" else x.astype(np.float32)
    passes = 8 if prec == "f64" else 4
    plan = hsvd.Plan(700, 520, 128, 128, "fixed_k", k, prec=prec)
    with pytest.raises(hsvd.HsvdError):
        plan.refine(1, 0.0)                                    # no run yet: ENOTREADY
    plan.run([to_device(xin, prec)])
    it, err = plan.refine(passes, 0.0)
    assert it == passes and err >= 0.0
    got = plan.factors(0)
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0
    res = oracle_run(xin, 128, 128, "fixed_k", k, prec)
    ref = oracle.iterative_improvement(np.asarray(xin, np.float64), res.v, res.s, eps=0.0, max_iters=passes,
                                       rank_tol=RANK_TOL[prec])
    check(xin, got, ref, prec, f"refine {prec}", s_true=s_true)
    # both sit on the truncated SVD (the power iteration's fixed point)
    ut, stt, vt = H.truncated_svd(np.asarray(xin, np.float64), k)
    assert oracle.sigma_rel_err(got[1], stt, k) <= TOL[prec][0]


def test_refine_stopping_rule_and_error_drop():
    """'while Error > eps': a huge eps stops after one pass, eps = 0 runs
    them all; on a gamma-truncated result the error against the truncated
    SVD drops (Section 4)."""
    s_true = 0.9 ** np.arange(60)
    x = W.planted(400, 320, s_true, noise=1e-4, tag=102).astype(np.float32)
    plan = hsvd.Plan(400, 320, 100, 80, "gamma", 0.05, rank_cap=64, prec="f32", power_iters=4)
    xd = torch.from_numpy(x).cuda()
    plan.run([xd])
    u0, s0, v0 = plan.factors(0)
    r = s0.size
    ut, st, vt = H.truncated_svd(x.astype(np.float64), r)
    xk = (ut * st) @ vt.T
    before = H.relative_error(xk, (u0.astype(np.float64) * s0) @ v0.T.astype(np.float64))
    assert plan.refine(5, 1e9)[0] == 1
    plan.run([xd])
    it, err = plan.refine(20, 1e-3)
    assert 1 <= it <= 20 and (err <= 1e-3 or it == 20)
    u1, s1, v1 = plan.factors(0)
    after = H.relative_error(xk, (u1.astype(np.float64) * s1) @ v1.T.astype(np.float64))
    assert before > 1e-4 and after < 0.8 * before, (before, after)
    plan.run([xd])
    assert plan.refine(4, 0.0)[0] == 4


# ---------------------------------------------------------------- graph replay and timing modes

def test_graph_replay_equals_step_launches_and_timing_modes():
    """Untimed runs replay a CUDA graph of the launch list; timed runs launch
    step by step (mode 1) or through a graph with events around the core
    SVDs (mode 2).  The kernels and their order are the same, so the factors
    are bitwise identical; mode 2 reports only the core-SVD steps."""
    x = W.exp_decay(1024, 768, r=200, noise=1e-5, tag=111, dtype=np.float32)
    xd = torch.from_numpy(x).cuda()
    plan = hsvd.Plan(1024, 768, 256, 256, "fixed_k", 24, prec="bf16_mixed", power_iters=1)
    outs = []
    for mode in (0, 1, 2, 0):
        plan.set_timing(mode)
        plan.run([xd])
        outs.append(plan.factors(0))
        t, runs = plan.step_times()
        kinds = [s["kind"] for s in plan.steps()]
        if mode == 1:
            assert runs == 1 and all(v > 0 for v in t)
        if mode == 2:
            assert runs == 1
            bad = [(i, k, v) for i, (v, k) in enumerate(zip(t, kinds)) if (v > 0) != (k == "jacobi")]
            assert not bad, bad
    plan.set_timing(0)
    for u, s, v in outs[1:]:
        assert np.array_equal(u, outs[0][0]) and np.array_equal(s, outs[0][1]) and np.array_equal(v, outs[0][2])


# ---------------------------------------------------------------- tall-skinny blocks, gamma rule (the paper's sweeps)

@pytest.mark.parametrize("bc", [8, 16, 64])
@pytest.mark.parametrize("prec", ["f32", "bf16_mixed"])
def test_gamma_tall_skinny_blocks(bc, prec):
    """The paper's experiments cut CFD snapshot matrices (m x 1024, m ~ 1e5)
    into tall blocks only 8-64 columns wide and truncate with gamma = 1e-2
    (Section 4).  A quarter-size stand-in (33025 x 256, a ragged last slab)
    with a decaying spectrum that leaves ~28 modes above gamma: many narrow
    blocks, many small merges."""
    s_true = np.exp(-np.arange(60) / 6.0)
    x = W.planted(33025, 256, s_true, noise=1e-6, tag=120 + bc).astype(np.float32)
    xin = W.bf16_round(x) if prec == "bf16_mixed" else x
    (got,), st, _ = run_gpu([xin], 8192, bc, "gamma", 1e-2, prec, rank_cap=64, power_iters=2)
    assert st["not_converged"] == 0 and st["nonfinite"] == 0
    ref = oracle_run(xin, 8192, bc, "gamma", 1e-2, prec, rank_cap=64)
    check(xin, got, ref, prec, f"gamma {bc}-wide {prec}", s_true=s_true)


# ---------------------------------------------------------------- the X^T X variant (Section 4)

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gram_variant(prec):
    """Section 4 also runs the method on X^T X of a tall snapshot matrix.
    hsvd_gram forms X^T X on the device (checked against the FP64 product);
    the method on it matches the oracle on the same Gram bytes, and its
    singular values are the squares of X's (top gap-separated modes)."""
    s_true = np.exp(-np.arange(80) / 8.0)
    x = W.planted(20000, 384, s_true, noise=1e-6, tag=140)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(x).to(dt).cuda()
    g = torch.empty((384, 384), dtype=dt, device="cuda")
    hsvd.hsvd_gram(xd, g)
    torch.cuda.synchronize()
    gh = g.cpu().numpy()
    xr = xd.cpu().numpy().astype(np.float64)
    exact = xr.T @ xr
    err = np.abs(gh - exact).max() / np.abs(exact).max()
    assert err <= (1e-14 if prec == "f64" else 2e-6), err
    # the paper's gamma = 1e-4 on X^T X (~1e-2 on X); FP32 cannot resolve
    # sigma ~ 1e-4 sigma_1 to 1e-4 relative, so its run keeps gamma = 1e-2
    gamma = 1e-4 if prec == "f64" else 1e-2
    (got,), st, _ = run_gpu([gh], 128, 64, "gamma", gamma, prec, rank_cap=64, power_iters=2)
    ref = oracle_run(gh, 128, 64, "gamma", gamma, prec, rank_cap=64)
    check(gh, got, ref, prec, f"gram {prec}", s_true=s_true ** 2)
    s_x = np.linalg.svd(xr, compute_uv=False)
    lead = 10  # sigma(G) >= 0.08 sigma_1: far above every truncation of the method
    assert np.allclose(got[1][:lead], s_x[:lead] ** 2, rtol=1e-6 if prec == "f64" else 1e-4, atol=0)


# ---------------------------------------------------------------- seeded sweep of shapes

def _sweep_cases():
    g = np.random.default_rng(20260102)
    cases = []
    for i in range(18):
        m = int(g.integers(40, 900))
        n = int(g.integers(40, 900))
        br = int(g.integers(16, max(17, m + 1)))
        bc = int(g.integers(16, max(17, n + 1)))
        if i % 2 == 1:  # multiples of 8: the tensor-core path of the mixed precision
            br, bc = max(8, br // 8 * 8), max(8, bc // 8 * 8)
        k = int(g.integers(1, 40))
        prec = ["f32", "bf16_mixed", "f64"][i % 3]
        tree = "row_then_col" if i % 4 == 1 else "col_then_row"
        cases.append((i, m, n, br, bc, k, prec, tree))
    return cases


@pytest.mark.parametrize("i,m,n,br,bc,k,prec,tree", _sweep_cases())
def test_seeded_shape_sweep(i, m, n, br, bc, k, prec, tree):
    """Random shapes, ragged grids, ranks and tree orders (seeded): exactly
    low-rank inputs of rank r <= k, so every truncation is lossless and the
    result must equal the oracle and the planted spectrum whatever the grid.
    (With r > k and no noise, a block whose k-th and (k+1)-th values nearly
    tie makes the kept subspace, and so the tail of the result, depend on
    rounding: such inputs have no unique answer to compare.)"""
    g = np.random.default_rng(1000 + i)
    r = int(min(m, n, g.integers(1, k + 1)))
    s_true = np.sort(g.uniform(0.5, 2.0, r))[::-1] * (0.7 ** np.arange(r))
    x = W.planted(m, n, s_true, noise=0.0, tag=2000 + i)
    if prec == "bf16_mixed":
        x = W.bf16_round(x.astype(np.float32))
    xin = x if prec == "f64" else np.asarray(x, np.float32)
    (got,), st, _ = run_gpu([xin], br, bc, "fixed_k", k, prec, tree=tree, power_iters=4, oversample=max(k, 16))
    assert st["nonfinite"] == 0
    ref = oracle_run(xin, br, bc, "fixed_k", k, prec, tree=tree)
    # BF16 storage adds a full-rank rounding term (~1e-3 of sigma_1 in norm):
    # the input is no longer exactly rank r, and only the planted values well
    # above that level are determined
    s_gate = s_true if prec != "bf16_mixed" else s_true[s_true >= 0.05 * s_true[0]]
    check(xin, got, ref, prec, f"sweep {i} {m}x{n}/{br}x{bc} k={k} r={r} {prec} {tree}", s_true=s_gate)


def _sweep_rule_cases():
    g = np.random.default_rng(20260103)
    cases = []
    for i in range(9):
        mode = ["gamma", "energy"][i % 2]
        prec = ["f32", "bf16_mixed", "f64"][i % 3]
        sizes = [(int(g.integers(64, 700)), int(g.integers(64, 700))) for _ in range(1 + i % 3)]
        br, bc = int(g.integers(32, 300)), int(g.integers(32, 300))
        if prec == "bf16_mixed" and i % 2:
            br, bc = br // 8 * 8, bc // 8 * 8
        cases.append((i, mode, prec, sizes, br, bc))
    return cases


@pytest.mark.parametrize("i,mode,prec,sizes,br,bc", _sweep_rule_cases())
def test_seeded_rule_and_batch_sweep(i, mode, prec, sizes, br, bc):
    """Gamma and energy rules on batches of 1-3 uneven matrices (seeded): a
    planted spectrum with a factor-1000 drop after r1 values plus 1e-6 noise,
    so each rule's decision is far from its threshold and unique."""
    g = np.random.default_rng(3000 + i)
    xs, trues = [], []
    for j, (m, n) in enumerate(sizes):
        r1 = int(g.integers(2, 12))
        top = np.sort(g.uniform(0.5, 2.0, r1))[::-1] * (0.85 ** np.arange(r1))
        s_true = np.concatenate([top, 1e-3 * top[-1] * 0.5 ** np.arange(6)])
        x = W.planted(m, n, s_true, noise=1e-6, tag=4000 + 10 * i + j)
        if prec == "bf16_mixed":
            x = W.bf16_round(x.astype(np.float32))
        xs.append(x if prec == "f64" else np.asarray(x, np.float32))
        trues.append(top)
    param = 1e-2 if mode == "gamma" else 0.999
    outs, st, _ = run_gpu(xs, br, bc, mode, param, prec, rank_cap=32, power_iters=4)
    assert st["nonfinite"] == 0
    for x, got, top in zip(xs, outs, trues):
        ref = oracle_run(x, br, bc, mode, param, prec, rank_cap=32)
        check(x, got, ref, prec, f"rules {i} {mode} {prec} {x.shape}/{br}x{bc}", s_true=top)


# ---------------------------------------------------------------- limits of the planner

@pytest.mark.parametrize("m,n,br,bc,k,prec", [
    (640, 512, 320, 256, 100, "f64"),          # 200-wide FP64 sketches and cores (global-memory kernels)
    (1024, 1024, 512, 512, 128, "bf16_mixed"),  # 256-wide tensor-core operands, 256 x 256 cores on clusters
    (1, 300, 1, 64, 1, "f32"),                  # one row
    (300, 1, 64, 1, 1, "f32"),                  # one column
    (5, 7, 2, 3, 2, "f32"),                     # 3 x 3 grid of 2 x 3 blocks, ragged
    (50, 40, 64, 64, 60, "f32"),                # k above min(m, n), one partial block
])
def test_planner_limits(m, n, br, bc, k, prec):
    r = min(m, n, 20)
    s_true = 0.8 ** np.arange(r)
    x = W.planted(m, n, s_true, noise=0.0, tag=5000 + m + n)
    if prec == "bf16_mixed":
        x = W.bf16_round(x.astype(np.float32))
    xin = x if prec == "f64" else np.asarray(x, np.float32)
    (got,), st, _ = run_gpu([xin], br, bc, "fixed_k", k, prec, power_iters=4)
    assert st["nonfinite"] == 0 and st["not_converged"] == 0
    ref = oracle_run(xin, br, bc, "fixed_k", k, prec)
    gate = s_true if prec != "bf16_mixed" else s_true[s_true >= 0.05]
    check(xin, got, ref, prec, f"limits {m}x{n}/{br}x{bc} k={k} {prec}", s_true=gate)


def test_autotune_picks_measured_variants_and_keeps_parity():
    """hsvd_options.autotune: the first run times the candidate kernels of
    each core-SVD launch and the pipeline depths of each tensor-core product,
    keeps the fastest, and the result still matches the oracle; later runs
    replay the same choices (bitwise-identical factors)."""
    x = W.exp_decay(1024, 1024, r=300, noise=1e-5, tag=71, dtype=np.float32)
    plan = hsvd.Plan(1024, 1024, 256, 256, "fixed_k", 64, prec="bf16_mixed", power_iters=1, autotune=True)
    xd = torch.from_numpy(x).cuda()
    plan.run([xd])
    u1, s1, v1 = plan.factors(0)
    tuned = [v for v in plan.variants() if v[2] > 1]
    assert any(v[1].startswith("jacobi:") for v in tuned), tuned
    assert any(v[1].startswith("tc_gemm:") for v in tuned), tuned
    plan.run([xd])
    u2, s2, v2 = plan.factors(0)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(u1, u2)
    xb = W.bf16_round(x)
    ref = oracle_run(xb, 256, 256, "fixed_k", 64, "bf16_mixed")
    check(xb, (u1, s1, v1), ref, "bf16_mixed", "autotuned", s_true=np.exp(-np.arange(300) / 20.0))
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0 and st["tensor_timeouts"] == 0


@pytest.mark.parametrize("k", [16, 48])
def test_tensor_core_wait_timeout_is_reported_and_the_context_survives(tmp_path, k):
    """The bounded waits of the tensor-core kernels: a test-only limit
    (HSVD_TC_FIRST_WAIT_CYCLES, read once per process) makes the MMA issuer's
    first wait give up before its tiles land; the kernel sets the error word,
    its other roles give up their waits, it waits for its own copies and
    MMAs, frees its tensor memory and returns.  k = 16: the input products
    (k_tc_gemm); k = 48: also the FP32-grade factor products (k_tcf, k_tcf2),
    wider than the skinny kernels' 32.  Run in a child process: the run
    reports tensor_timeouts > 0 and the CUDA context stays usable (a plain
    FP32 plan afterwards matches the oracle)."""
    import subprocess
    import sys
    code = f"""
import sys, numpy as np, torch
sys.path.insert(0, {ROOT_REPO!r})
from paper_1710_02812_gb300 import hsvd, workloads as W
import oracle
x = W.exp_decay(512, 512, r=100, noise=1e-5, tag=81, dtype=np.float32)
xd = torch.from_numpy(x).cuda()
p = hsvd.Plan(512, 512, 256, 256, "fixed_k", {k}, prec="bf16_mixed", power_iters=1)
p.run([xd])
st = p.status()
assert st["tensor_timeouts"] > 0, st
q = hsvd.Plan(512, 512, 256, 256, "fixed_k", 16, prec="f32", power_iters=1)
q.run([xd])
u, s, v = q.factors(0)
ref = oracle.hmat_svd(x.astype(np.float64), 256, 256, oracle.Rule("fixed_k", 16, rank_tol=1e-5))
assert s.size == 16 and oracle.sigma_rel_err(s, ref.s, 4) <= 1e-4  # the context still computes
torch.cuda.synchronize()
print("ok", st["tensor_timeouts"])
"""
    env = dict(os.environ, HSVD_TC_FIRST_WAIT_CYCLES="1")
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    assert p.stdout.strip().startswith("ok")
