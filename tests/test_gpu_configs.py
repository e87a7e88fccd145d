"""The five workload configurations at their full sizes, through the C ABI.

* 512^2 FP64 (k = 10): tests/test_gpu_parity.py, test_fp64_fixed_rank_512_parity.
* 8192^2 FP32 exp-decay (k = 64): FP32 and BF16-mixed paths against the
  oracle, element by element (the oracle finishes it in ~20 s).
* 32768 x 16384 POD-like BF16 snapshots (k = 64) and 65536^2 FP32 power-law
  (k = 128): the oracle cannot run them, so they are checked through
  properties that hold at any size, each a consequence of the method or of
  the construction, not a restatement of the code:
    - U and V have orthonormal columns;
    - the recovery step makes X V = U S exactly (Section 3: U S W^T = X V_r),
      so ||X V - U S|| is a rounding residue;
    - U S V^T = X V V^T is an orthogonal projection of X, so
      ||X - U S V^T||_F^2 = ||X||_F^2 - ||S||_F^2 (Pythagoras);
    - Weyl: every singular value of X lies within ||N||_2 of the noise-free
      part's (known exactly: s for the planted matrix, the singular values of
      the coefficient matrix for the POD snapshots, whose modes are
      orthonormal), ||N||_2 <= noise (sqrt(m) + sqrt(n)) (1 + 5%), so the
      leading computed sigma must sit in those bands;
    - Ritz residuals rho_i = ||X^T u_i - sigma_i v_i||: with X v_i = sigma_i u_i,
      z = [u_i; v_i] / sqrt(2) has residual rho_i / sqrt(2) for the Hermitian
      dilation [[0, X], [X^T, 0]], whose positive eigenvalues are the singular
      values of X.  Where Weyl's bands show that no other singular value of X
      lies within delta_i of sigma_i, the Kato-Temple bound gives
      |sigma_i - sigma_i(X)| <= (rho_i^2 / 2) / delta_i: a certified relative
      error, required <= 1e-4 (the accuracy target) for every mode it covers.
* 256 ragged FP32 matrices, 99.9% energy rule capped at 128: the whole batch in
  one plan; properties for every matrix and element-wise oracle parity for a
  sample of three matrices (the smallest), copied back to the host.
"""
import gc

import numpy as np
import pytest
import torch

import oracle
from oracle import hmat as H
from paper_1710_02812_gb300 import hsvd
from paper_1710_02812_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    torch.backends.cuda.matmul.allow_tf32 = False
    yield
    gc.collect()
    torch.cuda.empty_cache()


def device_factors(plan, idx=0):
    k = plan.kcap
    m, n = plan.m[idx], plan.n[idx]
    U = torch.empty((k, m), dtype=torch.float32, device="cuda")
    S = torch.empty(k, dtype=torch.float32, device="cuda")
    V = torch.empty((k, n), dtype=torch.float32, device="cuda")
    r = plan.factors_device(U, S, V, idx)
    return U[:r].t(), S[:r], V[:r].t()


def properties(x, U, S, V, chunk=4096):
    """Any-size checks of one result (x: the method's input as FP32 on the device)."""
    r = S.numel()
    eye = torch.eye(r, device="cuda")
    out = {"rank": r,
           "orth_u": float((U.t() @ U - eye).abs().max()),
           "orth_v": float((V.t() @ V - eye).abs().max())}
    out["recovery"] = float(torch.linalg.norm(x @ V - U * S) / torch.linalg.norm(S))
    out["rho"] = (torch.linalg.norm(x.t() @ U - V * S, dim=0) / S).cpu().numpy()
    x2 = res2 = 0.0
    for r0 in range(0, x.shape[0], chunk):
        xb = x[r0:r0 + chunk]
        x2 += float((xb.double() ** 2).sum())
        res2 += float(((xb - (U[r0:r0 + chunk] * S) @ V.t()).double() ** 2).sum())
    out["pythagoras"] = abs(res2 - (x2 - float((S.double() ** 2).sum()))) / x2
    out["rel_err"] = (res2 / x2) ** 0.5
    return out


def assert_properties(p, label, orth_tol, rec_tol):
    assert p["orth_u"] <= orth_tol and p["orth_v"] <= orth_tol, f"{label}: orthonormality {p}"
    assert p["recovery"] <= rec_tol, f"{label}: ||XV - US|| / ||S|| = {p['recovery']:.3e}"
    # exact for orthonormal U, V; first order in their orthonormality defects
    ptol = 3.0 * (p["orth_u"] + p["orth_v"]) + 1e-5
    assert p["pythagoras"] <= ptol, f"{label}: Pythagoras defect {p['pythagoras']:.3e} > {ptol:.3e}"


def weyl_band(sig, s_free, nb, upto):
    """sigma_i(X) lies within nb >= ||X - X_free||_2 of s_free[i] (Weyl)."""
    d = np.abs(sig[:upto] - s_free[:upto])
    assert np.all(d <= nb + 1e-4 * s_free[:upto]), f"outside the Weyl band {nb:.3e}: {d.max():.3e}"


def certified_rel_err(sig, rho_rel, s_free, nb, upto):
    """Kato-Temple bounds on |sigma_i - sigma_i(X)| / sigma_i for i < upto
    (nan where the Weyl bands cannot separate sigma_i from its neighbours)."""
    out = np.full(upto, np.nan)
    free = np.concatenate([s_free, [0.0]])        # 0: the cluster of the noise-level values
    for i in range(upto):
        others = np.delete(free, i)
        delta = np.min(np.maximum(np.abs(sig[i] - others) - nb, 0.0))
        r2 = (rho_rel[i] * sig[i]) ** 2 / 2.0
        if delta > np.sqrt(r2):
            out[i] = r2 / delta / sig[i]
    return out


def assert_certified(sig, rho_rel, s_free, nb, upto, need):
    b = certified_rel_err(sig, rho_rel, s_free, nb, upto)
    ok = ~np.isnan(b)
    assert ok.sum() >= need, f"only {ok.sum()} modes certifiable: {b}"
    assert np.all(b[ok] <= 1e-4), f"certified sigma errors {b[ok]}"
    return b


# ---------------------------------------------------------------- 8192^2 exp-decay (element-wise vs oracle)

@pytest.mark.parametrize("prec", ["f32", "bf16_mixed"])
def test_exp_decay_8192_against_oracle(prec):
    x, cfg = W.exp_decay_8192()
    xin = W.bf16_round(x) if prec == "bf16_mixed" else x   # the mixed path computes on BF16 values
    plan = hsvd.Plan(8192, 8192, 512, 512, "fixed_k", 64, prec=prec, power_iters=1)
    plan.run([torch.from_numpy(x).cuda()])
    u, s, v = plan.factors(0)
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0 and st["tensor_timeouts"] == 0
    ref = H.hmat_svd(xin.astype(np.float64), 512, 512, H.Rule("fixed_k", 64, rank_cap=64, rank_tol=1e-5))
    s_true = np.exp(-np.arange(512) / 20.0)
    j = oracle.gap_prefix(s_true, 64)
    assert s.size == 64 and j == 64
    err = oracle.sigma_rel_err(s, ref.s, j)
    ang_u = oracle.leading_subspace_angle(u, ref.u, ref.s, upto=j)
    ang_v = oracle.leading_subspace_angle(v, ref.v, ref.s, upto=j)
    assert err <= 1e-4 and ang_u <= 1e-3 and ang_v <= 1e-3, (err, ang_u, ang_v)


# ---------------------------------------------------------------- 32768 x 16384 POD snapshots (BF16)

def test_pod_snapshots_32768x16384_bf16_properties():
    stats = {}
    x, c = W.pod_fourier_device(stats=stats)
    m, n = x.shape
    plan = hsvd.Plan(m, n, 1024, 1024, "fixed_k", 64, prec="bf16_mixed", in_dtype="bf16", power_iters=1)
    plan.run([x])
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0 and st["tensor_timeouts"] == 0
    assert st["min_rank"] == st["max_rank"] == 64
    U, S, V = device_factors(plan)
    xf = x.float()
    p = properties(xf, U, S, V)
    assert_properties(p, "pod", orth_tol=2e-3, rec_tol=5e-4)
    sig = S.cpu().numpy().astype(np.float64)
    s_free = np.linalg.svd(c, compute_uv=False)          # the modes are orthonormal
    # ||N||_2 <= noise (sqrt m + sqrt n) (+5%); the BF16 storage rounding R of
    # the FP32 snapshots adds at most ||R||_F (measured by the generator)
    nb = 1.05 * 1e-3 * (np.sqrt(m) + np.sqrt(n)) + stats["rounding_fro"]
    lead = int(np.sum(s_free > 10 * nb))                   # modes well above the noise
    assert lead >= 4
    weyl_band(sig, s_free, nb, lead)
    assert_certified(sig, p["rho"], s_free, nb, lead, need=4)
    del plan, x, xf
    gc.collect()
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- 65536^2 power law (k = 128)

@pytest.mark.parametrize("prec", ["f32", "bf16_mixed"])
def test_power_law_65536_properties(prec):
    x, cfg = W.power_law_65536()
    m, n = x.shape
    plan = hsvd.Plan(m, n, 1024, 1024, "fixed_k", 128, prec=prec, power_iters=1)
    plan.run([x])
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0 and st["tensor_timeouts"] == 0
    assert st["min_rank"] == st["max_rank"] == 128
    U, S, V = device_factors(plan)
    plan.close()
    del plan
    gc.collect()
    torch.cuda.empty_cache()
    rounding = 0.0
    if prec == "bf16_mixed":
        xb = x.to(torch.bfloat16).float()                 # the values the mixed path computes on
        rounding = float(torch.linalg.norm(xb - x))
        del x
        x = xb
    p = properties(x, U, S, V)
    assert_properties(p, f"power law {prec}", orth_tol=1e-3, rec_tol=1e-5 if prec == "f32" else 5e-4)
    sig = S.cpu().numpy().astype(np.float64)
    nb = 1.05 * 1e-6 * (np.sqrt(m) + np.sqrt(n)) + 1e-6   # noise, plus FP32 storage of the product
    if prec == "bf16_mixed":
        nb += rounding                                      # ||X_bf16 - X||_F
    lead = int(np.sum(cfg["s"] > 10 * nb))
    assert lead >= 10
    weyl_band(sig, cfg["s"], nb, lead)
    assert_certified(sig, p["rho"], cfg["s"], nb, lead, need=6)
    # the paper reports errors of a few percent against the optimal rank-k error
    opt = np.sqrt(np.sum(cfg["s"][128:] ** 2) + 1e-12 * m * n) / np.sqrt(np.sum(cfg["s"] ** 2) + 1e-12 * m * n)
    assert p["rel_err"] <= 1.05 * opt, (p["rel_err"], opt)
    del x, U, S, V
    gc.collect()
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- 256 ragged matrices, energy 99.9%, cap 128

def test_ragged_batch_256_energy_rule():
    mats, sizes = W.ragged_batch_device()
    ms, ns = [s[0] for s in sizes], [s[1] for s in sizes]
    assert all(v % 1024 for v in ms + ns)
    plan = hsvd.Plan(ms, ns, 1024, 1024, "energy", 0.999, rank_cap=128, prec="f32", power_iters=1)
    plan.run(mats)
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0
    for i in range(len(mats)):                                 # every matrix: any-size properties
        U, S, V = device_factors(plan, i)
        p = properties(mats[i], U, S, V)
        assert_properties(p, f"batch[{i}] {sizes[i]}", orth_tol=2e-3, rec_tol=1e-5)
    order = np.argsort([m * n for m, n, _ in sizes])[:3]       # sample: the three smallest matrices
    for i in order:
        m, n, r = sizes[i]
        x = mats[i].cpu().numpy()
        u, s, v = plan.factors(int(i))
        ref = H.hmat_svd(x.astype(np.float64), 1024, 1024, H.Rule("energy", 0.999, rank_cap=128, rank_tol=1e-5))
        assert s.size == ref.s.size, (i, s.size, ref.s.size)
        # sigma normwise; the planted modes well above the noise element-wise
        assert float(np.max(np.abs(s - ref.s)) / ref.s[0]) <= 1e-2
        s_true = np.exp(-np.arange(r) / r) / r
        nb = 1e-4 * (np.sqrt(m) + np.sqrt(n))
        s_sig = s_true[s_true > 10 * nb]
        if s_sig.size:
            j = oracle.gap_prefix(s_sig, s_sig.size)
            if j:
                assert oracle.sigma_rel_err(s, ref.s, j) <= 1e-4
                assert oracle.leading_subspace_angle(u, ref.u, ref.s, upto=j) <= 1e-3
        xd = x.astype(np.float64)
        rg = np.linalg.norm(xd - (u.astype(np.float64) * s) @ v.T.astype(np.float64)) / np.linalg.norm(xd)
        ro = np.linalg.norm(xd - (ref.u * ref.s) @ ref.v.T) / np.linalg.norm(xd)
        assert abs(rg - ro) <= 0.01 * ro + 50 * 6e-8, (rg, ro)
