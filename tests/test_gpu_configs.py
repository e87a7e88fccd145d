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


def ritz_pairs(x, U, S, V, upto, chunk=4096):
    """For the first `upto` computed triplets, in FP64: theta_i = u_i^T X v_i
    (u_i, v_i normalised) and the residual norm eps_i of z = [u_i; v_i]/sqrt(2)
    for the Hermitian dilation H = [[0, X], [X^T, 0]]:
    eps_i^2 = (||X v_i - theta_i u_i||^2 + ||X^T u_i - theta_i v_i||^2) / 2.
    No identity of the method (X v = sigma u) is assumed."""
    u = U[:, :upto].double()
    v = V[:, :upto].double()
    u = u / torch.linalg.norm(u, dim=0)
    v = v / torch.linalg.norm(v, dim=0)
    xv = torch.empty_like(u)
    xtu = torch.zeros_like(v)
    for r0 in range(0, x.shape[0], chunk):
        xb = x[r0:r0 + chunk].double()
        xv[r0:r0 + chunk] = xb @ v
        xtu += xb.t() @ u[r0:r0 + chunk]
    theta = (u * xv).sum(0)
    e1 = torch.linalg.norm(xv - u * theta, dim=0)
    e2 = torch.linalg.norm(xtu - v * theta, dim=0)
    eps = torch.sqrt((e1 ** 2 + e2 ** 2) / 2)
    return theta.cpu().numpy(), eps.cpu().numpy()


def certified_sigma_errors(sig, theta, eps, s_free, nb):
    """Certified bounds on |sigma_i - sigma_i(X)| / sigma_i (nan where none).

    Weyl puts sigma_j(X) in [s_free_j - nb, s_free_j + nb] (and every value
    past the planted ones in [0, nb]).  Where theta_i lies strictly between the
    bands of its neighbours, the interval (alpha, beta) between those bands
    holds exactly one eigenvalue of the dilation, sigma_i(X), and Kato-Temple
    gives |theta_i - sigma_i(X)| <= eps_i^2 / min(theta_i - alpha, beta - theta_i).
    The returned sigma_i is then within |sigma_i - theta_i| of theta_i."""
    upto = theta.size
    free = np.concatenate([s_free, [0.0]])
    out = np.full(upto, np.nan)
    for i in range(upto):
        alpha = free[i + 1] + nb if i + 1 < free.size else nb
        beta = free[i - 1] - nb if i > 0 else np.inf
        delta = min(theta[i] - alpha, beta - theta[i])
        if not delta > 0:
            continue
        out[i] = (abs(sig[i] - theta[i]) + eps[i] ** 2 / delta) / sig[i]
    return out


def assert_certified(sig, theta, eps, s_free, nb, upto, need):
    """Every certifiable mode among the first `upto` within 1e-4 (the accuracy
    target), at least `need` of them certifiable; and the returned sigma_i
    agrees with its own Rayleigh quotient u_i^T X v_i to 1e-4."""
    rq = np.abs(sig[:upto] - theta[:upto]) / sig[:upto]
    assert np.all(rq <= 1e-4), f"|sigma_i - u_i^T X v_i| / sigma_i: {rq.max():.3e} at {rq.argmax()}"
    b = certified_sigma_errors(sig, theta[:upto], eps[:upto], s_free, nb)
    ok = ~np.isnan(b)
    assert ok.sum() >= need, f"only {ok.sum()} modes certifiable: {b}"
    assert np.all(b[ok] <= 1e-4), f"certified sigma errors {b[ok]}"
    return b


def spectral_norm_estimate(apply_gram, n, device, iters=40, seed=7):
    """||R||_2 from `iters` steps of the power method on R^T R (apply_gram(v)
    returns R^T R v, FP64), started from a seeded Gaussian block of 4 vectors
    (orthonormalised each step); the largest Ritz value of the last step.
    The power method approaches ||R||_2 from below; the callers multiply the
    estimate by a safety factor of 1.5."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    q = torch.randn((n, 4), generator=g, device=device, dtype=torch.float64)
    q, _ = torch.linalg.qr(q)
    lam = 0.0
    for _ in range(iters):
        z = apply_gram(q)
        lam = float(torch.linalg.eigvalsh(q.t() @ z).max())
        q, _ = torch.linalg.qr(z)
    return lam ** 0.5


def rounding_gram(x, chunk=4096):
    """v -> R^T R v for R = bf16(x) - x, formed chunk by chunk (R is never stored)."""
    def apply(v):
        out = torch.zeros_like(v)
        for r0 in range(0, x.shape[0], chunk):
            xb = x[r0:r0 + chunk]
            rc = (xb.to(torch.bfloat16).float() - xb).double()
            out += rc.t() @ (rc @ v)
        return out
    return apply


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
    x, c = W.pod_fourier_device(stats=stats, keep_rounding=True)
    m, n = x.shape
    plan = hsvd.Plan(m, n, 1024, 1024, "fixed_k", 64, prec="bf16_mixed", in_dtype="bf16", power_iters=1)
    plan.run([x])
    st = plan.status()
    assert st["not_converged"] == 0 and st["nonfinite"] == 0 and st["tensor_timeouts"] == 0
    assert st["min_rank"] == st["max_rank"] == 64
    U, S, V = device_factors(plan)
    del plan
    xf = x.float()
    p = properties(xf, U, S, V)
    assert_properties(p, "pod", orth_tol=2e-3, rec_tol=1e-5)
    sig = S.cpu().numpy().astype(np.float64)
    s_free = np.linalg.svd(c, compute_uv=False)          # the modes are orthonormal
    # ||X - X_free||_2 <= ||N||_2 + ||R||_2 + construction: the noise by
    # noise (sqrt m + sqrt n) (+5%); the BF16 storage rounding R of the FP32
    # snapshots by 1.5 x its power-method estimate; the FP32 construction of
    # phi C (entries relatively exact to ~1e-7) by 1e-5 sigma_1
    R = stats.pop("rounding")
    r2 = spectral_norm_estimate(lambda v: R.t().double() @ (R.double() @ v), n, "cuda")
    del R
    nb = 1.05 * 1e-3 * (np.sqrt(m) + np.sqrt(n)) + 1.5 * r2 + 1e-5 * s_free[0]
    lead = int(np.sum(s_free > 10 * nb))                   # modes well above the noise
    assert lead >= 4
    weyl_band(sig, s_free, nb, lead)
    theta, eps = ritz_pairs(xf, U, S, V, lead)
    b = assert_certified(sig, theta, eps, s_free, nb, lead, need=4)
    print(f"pod: recovery {p['recovery']:.2e} rounding ||R||_2 ~ {r2:.2e} (||R||_F {stats['rounding_fro']:.2e}) "
          f"certified {np.nanmax(b):.2e} over {lead} modes")
    del x, xf
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
    # ||X - X_free||_2: the noise, noise (sqrt m + sqrt n) (+5%), plus 1e-6 for
    # the FP32 storage of the product
    nb = 1.05 * 1e-6 * (np.sqrt(m) + np.sqrt(n)) + 1e-6
    if prec == "bf16_mixed":
        # the mixed path computes on the BF16-rounded values: their rounding R
        # enters with 1.5 x its power-method estimate of ||R||_2
        r2 = spectral_norm_estimate(rounding_gram(x), n, "cuda")
        nb += 1.5 * r2
        x = x.to(torch.bfloat16).float()                   # the values the path computed on
        gc.collect()
        torch.cuda.empty_cache()
    p = properties(x, U, S, V)
    assert_properties(p, f"power law {prec}", orth_tol=1e-3, rec_tol=1e-5)
    sig = S.cpu().numpy().astype(np.float64)
    lead = int(np.sum(cfg["s"] > 10 * nb))
    assert lead >= 10
    weyl_band(sig, cfg["s"], nb, lead)
    theta, eps = ritz_pairs(x, U, S, V, lead)
    b = assert_certified(sig, theta, eps, cfg["s"], nb, lead, need=6)
    print(f"power law {prec}: recovery {p['recovery']:.2e} nb {nb:.2e} certified {np.nanmax(b):.2e} over "
          f"{int(np.sum(~np.isnan(b)))} of {lead} modes")
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
    # sample: the three smallest matrices among those with at least four
    # planted modes well above the noise edge (s_i > 5 noise (sqrt m + sqrt n)),
    # so the element-wise sigma and angle gates run on every sampled matrix
    def n_signal(m, n, r):
        return int(np.sum(np.exp(-np.arange(r) / r) / r > 5 * 1e-4 * (np.sqrt(m) + np.sqrt(n))))
    eligible = [i for i, (m, n, r) in enumerate(sizes) if n_signal(m, n, r) >= 4]
    assert len(eligible) >= 3
    order = sorted(eligible, key=lambda i: sizes[i][0] * sizes[i][1])[:3]
    for i in order:
        m, n, r = sizes[i]
        x = mats[i].cpu().numpy()
        u, s, v = plan.factors(int(i))
        ref = H.hmat_svd(x.astype(np.float64), 1024, 1024, H.Rule("energy", 0.999, rank_cap=128, rank_tol=1e-5))
        assert s.size == ref.s.size, (i, s.size, ref.s.size)
        # sigma normwise; the planted modes well above the noise element-wise
        assert float(np.max(np.abs(s - ref.s)) / ref.s[0]) <= 1e-2
        s_true = np.exp(-np.arange(r) / r) / r
        s_sig = s_true[:n_signal(m, n, r)]
        j = oracle.gap_prefix(s_sig, s_sig.size)
        assert j >= 4, (i, sizes[i], j)
        assert oracle.sigma_rel_err(s, ref.s, j) <= 1e-4
        assert oracle.leading_subspace_angle(u, ref.u, ref.s, upto=j) <= 1e-3
        assert oracle.leading_subspace_angle(v, ref.v, ref.s, upto=j) <= 1e-3
        xd = x.astype(np.float64)
        rg = np.linalg.norm(xd - (u.astype(np.float64) * s) @ v.T.astype(np.float64)) / np.linalg.norm(xd)
        ro = np.linalg.norm(xd - (ref.u * ref.s) @ ref.v.T) / np.linalg.norm(xd)
        assert abs(rg - ro) <= 0.01 * ro + 50 * 6e-8, (rg, ro)
