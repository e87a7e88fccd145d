"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each checks a value that is
known independently (a planted spectrum, a closed form, an exact special case,
a bound, a library SVD on a case where the method is provably exact), chosen
so a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import Rule
from oracle import hmat as H
from paper_1710_02812_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

GRIDS = [  # (m, n, block_rows, block_cols): square, ragged, odd leaf counts,
           # row-only (one column slice) and column-only (one row slab) grids
    (64, 64, 64, 64),
    (64, 64, 32, 32),
    (70, 90, 24, 20),
    (60, 56, 60, 8),    # 1 x 7 grid: column tree with 7 leaves (Iwen-style)
    (60, 56, 9, 56),    # 7 x 1 grid: row tree only
    (50, 75, 10, 15),   # 5 x 5 grid
    (33, 47, 11, 16),   # 3 x 3 grid, ragged
]


def planted_exact(m, n, r, tag=0, s=None):
    if s is None:
        s = np.linspace(3.0, 0.5, r)
    a, u, s, v = W.planted(m, n, s, noise=0.0, tag=tag, return_factors=True)
    return a, u, s, v


# ---------------------------------------------------------------- rules

def test_rule_fixed_k_closed_form():
    s = np.array([5.0, 4.0, 3.0, 2.0, 1.0])
    assert Rule(H.FIXED_K, 3).rank(s) == 3
    assert Rule(H.FIXED_K, 9).rank(s) == 5           # cannot exceed what exists
    assert Rule(H.FIXED_K, 3, rank_cap=2).rank(s) == 2
    s0 = np.array([1.0, 1e-20, 0.0])
    assert Rule(H.FIXED_K, 3).rank(s0) == 1          # numerically zero dropped
    assert Rule(H.FIXED_K, 3).rank(np.zeros(4)) == 0
    assert Rule(H.FIXED_K, 3).rank(np.zeros(0)) == 0


def test_rule_gamma_is_non_strict():
    s = np.array([10.0, 5.0, 1.0, 0.999999, 0.5])
    assert Rule(H.GAMMA, 0.1).rank(s) == 3           # sigma_i >= 0.1 * 10 keeps 1.0
    assert Rule(H.GAMMA, 0.5).rank(s) == 2
    assert Rule(H.GAMMA, 0.01).rank(s) == 5


def test_rule_energy_closed_form():
    s = np.sqrt(np.array([50.0, 30.0, 15.0, 4.0, 1.0]))   # energies sum to 100
    assert Rule(H.ENERGY, 0.80).rank(s) == 2
    assert Rule(H.ENERGY, 0.95).rank(s) == 3
    assert Rule(H.ENERGY, 0.951).rank(s) == 4
    assert Rule(H.ENERGY, 1.0).rank(s) == 5
    # total larger than the values seen (energy outside the kept spectrum)
    assert Rule(H.ENERGY, 0.99).rank(s, total=200.0) == 5
    assert Rule(H.ENERGY, 0.41).rank(s, total=200.0) == 3
    assert Rule(H.ENERGY, 0.39).rank(s, total=200.0) == 2


# ---------------------------------------------------------------- tree

@pytest.mark.parametrize("count,levels", [(1, 0), (2, 1), (3, 2), (5, 3), (7, 3), (8, 3), (64, 6), (65, 7)])
def test_tree_levels_ceil_log2(count, levels):
    sched = H.tree_schedule(count)
    assert len(sched) == levels
    # every level pairs adjacent positions; the survivors shrink as ceil(n/2)
    n = count
    for lv in sched:
        assert lv == [(i, i + 1) for i in range(0, n - 1, 2)]
        n = (n + 1) // 2
    assert n == 1


def test_merge_tree_visits_every_leaf_once_and_carries_odd():
    seen = []

    def merge(a, b, level, idx):
        seen.append((level, idx))
        return a + b

    for count in (1, 2, 3, 5, 7, 11):
        seen.clear()
        out = H.merge_tree([[i] for i in range(count)], merge)
        assert out == list(range(count))           # order preserved, nothing lost
        assert len(seen) == count - 1               # P - 1 merges (Section 3.1)


# ---------------------------------------------------------------- exactness

@pytest.mark.parametrize("m,n,br,bc", GRIDS)
def test_exact_rank_inputs_recovered(m, n, br, bc):
    """Exactly rank-r input with r <= k: every truncation is lossless, so the
    method returns the planted spectrum and subspaces (Section 3 proofs)."""
    r = 4
    a, u, s, v = planted_exact(m, n, r, tag=m + n)
    for tree in ("col_then_row", "row_then_col"):
        res = H.hmat_svd(a, br, bc, Rule(H.FIXED_K, 6, rank_tol=1e-10), tree=tree)
        assert res.s.size == r
        np.testing.assert_allclose(res.s, s, rtol=1e-12)
        for i in range(r):
            assert oracle.principal_angle(res.u[:, i:i + 1], u[:, i:i + 1]) < 1e-10
            assert oracle.principal_angle(res.v[:, i:i + 1], v[:, i:i + 1]) < 1e-10
        np.testing.assert_allclose((res.u * res.s) @ res.v.T, a, atol=1e-12)


@pytest.mark.parametrize("m,n,br,bc", GRIDS)
def test_lossless_when_k_covers_everything(m, n, br, bc):
    """With k >= min(m, n) no truncation drops anything, so for ANY matrix the
    method is the full SVD; here checked on a dense random full-rank matrix."""
    g = np.random.default_rng(m * 1000 + n)
    a = g.standard_normal((m, n))
    res = H.hmat_svd(a, br, bc, Rule(H.FIXED_K, min(m, n), rank_tol=1e-13))
    s_ref = np.linalg.svd(a, compute_uv=False)
    np.testing.assert_allclose(res.s, s_ref, rtol=1e-10)
    np.testing.assert_allclose((res.u * res.s) @ res.v.T, a, atol=1e-10)


def test_one_by_one_grid_is_truncated_svd_planted():
    """A 1x1 grid is the textbook truncated SVD (Eckart-Young, Section 1):
    checked on a planted spectrum, so the expected values are known."""
    s = np.array([8.0, 4.0, 2.0, 1.0, 0.5, 0.25])
    a, u, _, v = W.planted(40, 30, s, tag=11, return_factors=True)
    res = H.hmat_svd(a, 40, 30, Rule(H.FIXED_K, 3))
    np.testing.assert_allclose(res.s, s[:3], rtol=1e-13)
    err2 = np.linalg.norm(a - (res.u * res.s) @ res.v.T) ** 2
    np.testing.assert_allclose(err2, np.sum(s[3:] ** 2), rtol=1e-10)


def test_diagonal_and_permuted_diagonal():
    """sigma of a (row- and column-permuted) diagonal matrix is sorted |d|;
    blocks share no rows/columns of support, so every merge is exact and the
    top-k survive all truncations."""
    g = np.random.default_rng(5)
    d = g.permutation(np.arange(1, 41, dtype=np.float64)) * g.choice([-1.0, 1.0], 40)
    a = np.zeros((48, 40))
    a[np.arange(40), np.arange(40)] = d
    a = a[g.permutation(48)][:, g.permutation(40)]
    expect = np.sort(np.abs(d))[::-1]
    for br, bc, k in [(48, 40, 5), (16, 8, 7), (7, 9, 12), (5, 40, 3), (48, 3, 10)]:
        res = H.hmat_svd(a, br, bc, Rule(H.FIXED_K, k))
        np.testing.assert_allclose(res.s, expect[:k], rtol=1e-13)
        # each singular vector is a signed unit coordinate vector
        assert np.allclose(np.sort(np.abs(res.u), axis=0)[-1], 1.0)
        assert np.allclose(np.sort(np.abs(res.v), axis=0)[-1], 1.0)


def test_repeated_values_rotation_invariant():
    """A cluster of equal singular values defines a subspace, not vectors;
    the subspace of the cluster must match the planted one."""
    s = np.array([5.0, 2.0, 2.0, 2.0, 1.0])
    a, u, _, v = W.planted(60, 50, s, tag=21, return_factors=True)
    res = H.hmat_svd(a, 20, 25, Rule(H.FIXED_K, 5))
    np.testing.assert_allclose(res.s, s, rtol=1e-12)
    assert oracle.principal_angle(res.u[:, 1:4], u[:, 1:4]) < 1e-10
    assert oracle.principal_angle(res.v[:, 1:4], v[:, 1:4]) < 1e-10


def test_outputs_orthonormal_on_noisy_input():
    a, cfg = W.fixed_rank_512()
    res = H.hmat_svd(a, cfg["block_rows"], cfg["block_cols"], Rule(H.FIXED_K, cfg["k"]))
    assert oracle.orthonormality_defect(res.u) < 1e-12
    assert oracle.orthonormality_defect(res.v) < 1e-12
    assert np.all(np.diff(res.s) <= 0)


def test_eckart_young_lower_bound_and_paper_error_claim():
    """For every grid the rank-k result cannot beat the best rank-k error
    sqrt(sum_{i>k} s_i^2) (planted s), and the paper's relative error to X_k
    is typically below 3% (abstract)."""
    s = 2.0 ** -np.arange(12, dtype=np.float64)
    a = W.planted(36, 30, s, tag=31)
    k = 4
    best = np.sqrt(np.sum(s[k:] ** 2))
    xk = (lambda t: (t[0] * t[1]) @ t[2].T)(H.truncated_svd(a, k))
    for br, bc in [(36, 30), (12, 10), (9, 6), (5, 7), (36, 3), (4, 30)]:
        res = H.hmat_svd(a, br, bc, Rule(H.FIXED_K, k))
        ahat = (res.u * res.s) @ res.v.T
        err = np.linalg.norm(a - ahat)
        assert err >= best * (1 - 1e-12)
        if (br, bc) == (36, 30):
            np.testing.assert_allclose(err, best, rtol=1e-10)
        assert H.relative_error(xk, ahat) < 0.03


def test_sibling_order_does_not_change_merge():
    g = np.random.default_rng(9)
    u1, _ = np.linalg.qr(g.standard_normal((40, 5)))
    u2, _ = np.linalg.qr(g.standard_normal((40, 4)))
    s1 = np.array([5.0, 3, 2, 1, 0.5])
    s2 = np.array([4.0, 2.5, 1.5, 0.2])
    rule = Rule(H.FIXED_K, 6)
    ua, sa = H.mat_merge(u1, s1, u2, s2, rule)
    ub, sb = H.mat_merge(u2, s2, u1, s1, rule)
    np.testing.assert_allclose(sa, sb, rtol=1e-13)
    assert oracle.principal_angle(ua, ub) < 1e-12


@pytest.mark.parametrize("overlap", [0, 2, 4])
def test_orthogonal_complement_merge_equals_plain_merge(overlap):
    """Eqs. orthmerge1/orthmerge (with R Sigma_2) reach the plain MAT result,
    including when U2 shares directions with U1 (rank-deficient Q)."""
    g = np.random.default_rng(100 + overlap)
    h = 50
    base, _ = np.linalg.qr(g.standard_normal((h, 12)))
    u1 = base[:, :5]
    # U2: `overlap` directions inside span(U1), the rest new
    rot, _ = np.linalg.qr(g.standard_normal((5, 5)))
    u2 = np.concatenate([(u1 @ rot)[:, :overlap], base[:, 5:5 + 4 - overlap]], axis=1)
    s1 = np.array([6.0, 4, 3, 1, 0.3])
    s2 = np.array([5.0, 2, 0.7, 0.1])
    for k in (3, 6, 9):
        rule = Rule(H.FIXED_K, k)
        up, sp = H.mat_merge(u1, s1, u2, s2, rule)
        uo, so, e = H.mat_merge_orth(u1, s1, u2, s2, rule, return_core=True)
        np.testing.assert_allclose(so, sp, rtol=1e-12)
        assert oracle.orthonormality_defect(uo) < 1e-12
        for g0, g1 in oracle.metrics.gap_groups(sp):
            assert oracle.principal_angle(uo[:, g0:g1], up[:, g0:g1]) < 1e-10
        assert e.shape == (5 + 4 - overlap, 9)


def test_printed_lower_right_block_would_be_caught():
    """Plant the printed form Sigma_2 R (reading 1) in a copy of the merge on
    the CPU: the comparison with the plain MAT must fail."""
    g = np.random.default_rng(3)
    u1, _ = np.linalg.qr(g.standard_normal((30, 4)))
    u2, _ = np.linalg.qr(g.standard_normal((30, 4)))
    s1 = np.array([4.0, 3, 2, 1])
    s2 = np.array([3.5, 1.5, 0.9, 0.4])
    p = u1.T @ u2
    q = u2 - u1 @ p
    uq, sq, vq = np.linalg.svd(q, full_matrices=False)
    r = sq[:, None] * vq
    e_bad = np.block([[np.diag(s1), p * s2[None, :]], [np.zeros((4, 4)), s2[:, None] * r]])
    s_bad = np.linalg.svd(e_bad, compute_uv=False)[:6]
    _, s_ok = H.mat_merge(u1, s1, u2, s2, Rule(H.FIXED_K, 6))
    assert np.max(np.abs(s_bad - s_ok) / s_ok) > 1e-3


def test_zero_blocks_and_zero_matrix():
    g = np.random.default_rng(4)
    a = np.zeros((40, 40))
    a[:20, :20] = g.standard_normal((20, 3)) @ g.standard_normal((3, 20))
    res = H.hmat_svd(a, 20, 20, Rule(H.FIXED_K, 5, rank_tol=1e-10))
    s_ref = np.linalg.svd(a[:20, :20], compute_uv=False)[:3]
    np.testing.assert_allclose(res.s, s_ref, rtol=1e-12)
    res0 = H.hmat_svd(np.zeros((30, 20)), 10, 10, Rule(H.FIXED_K, 4))
    assert res0.s.size == 0 and res0.u.shape == (30, 0) and res0.v.shape == (20, 0)


def test_gamma_mode_on_planted_spectrum():
    """gamma keeps sigma_i >= gamma sigma_1 of each block; on an exactly
    low-rank input the final rank is the count of planted s_i >= gamma s_1
    when every block sees the whole spectrum (1 x C grid, row slabs full)."""
    s = np.array([10.0, 6.0, 2.5, 0.8, 0.05])
    a = W.planted(40, 60, s, tag=41)
    res = H.hmat_svd(a, 40, 60, Rule(H.GAMMA, 0.1))
    assert res.s.size == 3
    np.testing.assert_allclose(res.s, s[:3], rtol=1e-12)


def test_energy_mode_uses_block_frobenius_energy():
    s = np.sqrt(np.array([60.0, 25.0, 10.0, 4.0, 1.0]))
    a = W.planted(30, 30, s, tag=51)
    assert H.hmat_svd(a, 30, 30, Rule(H.ENERGY, 0.85)).s.size == 2
    assert H.hmat_svd(a, 30, 30, Rule(H.ENERGY, 0.95)).s.size == 3
    assert H.hmat_svd(a, 30, 30, Rule(H.ENERGY, 0.99)).s.size == 4


def test_row_then_col_is_transpose_of_col_then_row():
    a, _ = W.fixed_rank_512()
    a = a[:200, :160]
    r1 = H.hmat_svd(a, 64, 48, Rule(H.FIXED_K, 8), tree="row_then_col")
    r2 = H.hmat_svd(a.T, 48, 64, Rule(H.FIXED_K, 8), tree="col_then_row")
    np.testing.assert_allclose(r1.s, r2.s, rtol=1e-14)
    np.testing.assert_allclose(np.abs(r1.u), np.abs(r2.v), atol=1e-12)


def test_projection_step_is_exact_svd_of_projection():
    """U_y S_y (V_r V_y)^T is the exact SVD of X V_r V_r^T (Section 3)."""
    g = np.random.default_rng(8)
    x = g.standard_normal((30, 20))
    vr, _ = np.linalg.qr(g.standard_normal((20, 5)))
    u, s, v = H.recover_left(x, vr)
    np.testing.assert_allclose((u * s) @ v.T, x @ vr @ vr.T, atol=1e-12)
    assert oracle.orthonormality_defect(u) < 1e-13
    assert oracle.orthonormality_defect(v) < 1e-13


def test_slab_step_right_vectors_not_left():
    """V_j must be the right singular vectors of U_j^T X_j (n-dimensional);
    using the left ones (k-dimensional) or skipping the re-SVD would break
    the rank-1 closed form below."""
    a = np.outer([1.0, 2.0, 2.0], [2.0, 0.0, 1.0, 2.0])   # sigma = 3 * 3
    u_j = np.array([[1.0], [2.0], [2.0]]) / 3.0
    v, s = H.slab_step(u_j, a, Rule(H.FIXED_K, 1))
    np.testing.assert_allclose(s, [9.0], rtol=1e-14)
    np.testing.assert_allclose(np.abs(v[:, 0]), np.array([2.0, 0, 1, 2]) / 3.0, atol=1e-14)


def test_golden_fixtures():
    with open(os.path.join(GOLDEN, "closed_form_cases.json")) as f:
        cases = json.load(f)
    assert cases
    for case in cases:
        a = np.array(case["matrix"], dtype=np.float64)
        rule = Rule(case["mode"], case["param"], rank_tol=1e-12)
        res = H.hmat_svd(a, case["block_rows"], case["block_cols"], rule)
        np.testing.assert_allclose(res.s, case["sigma"], rtol=1e-12, err_msg=case["name"])
        if "u_abs" in case:
            np.testing.assert_allclose(np.abs(res.u), np.array(case["u_abs"]), atol=1e-12)
        if "v_abs" in case:
            np.testing.assert_allclose(np.abs(res.v), np.array(case["v_abs"]), atol=1e-12)


# ---------------------------------------------------------------- Alg. 2 (iterative improvement)

def test_iterative_improvement_exact_rank_stops_after_one_pass():
    """On an exactly rank-r input the MAT result is already exact: one pass,
    Error at rounding level, the planted sigma and subspaces unchanged."""
    s_true = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    x, u0, s0, v0 = W.planted(96, 80, s_true, tag=91, return_factors=True)
    res = H.hmat_svd(x, 32, 16, Rule("fixed_k", 8, rank_cap=8, rank_tol=1e-12))
    ref = oracle.iterative_improvement(x, res.v, res.s, eps=1e-3, max_iters=10, rank_tol=1e-12)
    assert ref.iterations == 1 and ref.errors[0] < 1e-13
    assert np.allclose(ref.s, s_true, rtol=1e-12, atol=0)
    assert oracle.principal_angle(ref.u, u0) < 1e-10 and oracle.principal_angle(ref.v, v0) < 1e-10


def test_iterative_improvement_is_a_power_iteration_to_the_truncated_svd():
    """From a deliberately poor V_hat (the top-k right vectors rotated 30
    degrees into the tail) the passes converge to LAPACK's truncated SVD.
    Each pass multiplies by X and X^T once (one power step on X^T X), so the
    subspace error shrinks by (s_{k+1}/s_k)^2 per pass and the singular
    values, second order in it, by (s_{k+1}/s_k)^4: the pass-to-pass Error
    must fall at that rate."""
    k = 6
    s_true = np.concatenate([np.linspace(4.0, 2.0, k), 0.8 * np.linspace(1.0, 0.5, 10)])
    x, u0, s0, v0 = W.planted(120, 90, s_true, tag=92, return_factors=True)
    th = np.deg2rad(30.0)
    v_start = np.cos(th) * v0[:, :k] + np.sin(th) * v0[:, k:2 * k]
    v_start, _ = np.linalg.qr(v_start)
    ref = oracle.iterative_improvement(x, v_start, np.full(k, 1.0), eps=1e-15, max_iters=80)
    ut, st, vt = H.truncated_svd(x, k)
    assert np.allclose(ref.s, st, rtol=1e-10, atol=0)
    assert oracle.principal_angle(ref.u, ut) < 1e-8 and oracle.principal_angle(ref.v, vt) < 1e-8
    e = np.array(ref.errors[2:12])
    rate = np.exp(np.mean(np.diff(np.log(e))))
    expect = (s_true[k] / s_true[k - 1]) ** 4
    assert 0.5 * expect < rate < 1.5 * expect, (rate, expect)


def test_iterative_improvement_stopping_rule():
    """'while Error > eps': a huge eps stops after the first pass, eps = 0
    runs every allowed pass."""
    x = W.planted(64, 64, np.linspace(3, 1, 8), noise=1e-3, tag=93)
    res = H.hmat_svd(x, 32, 32, Rule("fixed_k", 4, rank_cap=4))
    assert oracle.iterative_improvement(x, res.v, res.s, eps=1e9, max_iters=7).iterations == 1
    assert oracle.iterative_improvement(x, res.v, res.s, eps=0.0, max_iters=7).iterations == 7


def test_iterative_improvement_reduces_the_mat_error():
    """Section 4: the error against the truncated SVD drops once iterative
    improvement is applied (here gamma truncation makes the MAT result
    visibly inexact)."""
    s_true = 0.9 ** np.arange(60)
    x = W.planted(200, 160, s_true, noise=1e-4, tag=94)
    rule = Rule("gamma", 0.05, rank_cap=64)
    res = H.hmat_svd(x, 50, 40, rule)
    r = res.s.size
    ut, st, vt = H.truncated_svd(x, r)
    xk = (ut * st) @ vt.T
    before = H.relative_error(xk, (res.u * res.s) @ res.v.T)
    ref = oracle.iterative_improvement(x, res.v, res.s, eps=1e-3, max_iters=20)
    after = H.relative_error(xk, (ref.u * ref.s) @ ref.v.T)
    assert before > 1e-4 and after < 0.8 * before, (before, after)


def test_trace_records_every_rank_decision_and_its_margin():
    """X = diag(10, 5, 1, 0.5) on a 2 x 2 grid, gamma = 0.1, derived by hand:
    the diagonal blocks keep both values (nearest to their thresholds 1 and
    0.1: 5 and 0.5, margin 0.4 of sigma_1), the off-diagonal blocks are zero
    (rank 0, no margin), each slab's merge and slab step repeat its block,
    and the row merge sees 10, 5, 1, 0.5 against the threshold 1: it keeps
    three and the deciding value 1 sits exactly on the threshold (margin 0,
    the tie a parity run must flag)."""
    x = np.diag([10.0, 5.0, 1.0, 0.5])
    res = oracle.hmat_svd(x, 2, 2, Rule("gamma", 0.1))
    names = [t[0] for t in res.trace.steps]
    ranks = [t[1] for t in res.trace.steps]
    margins = [t[2] for t in res.trace.steps]
    assert names == ["block0,0", "block0,1", "col0L0#0", "slab0",
                     "block1,0", "block1,1", "col1L0#0", "slab1", "rowL0#0"]
    assert ranks == [2, 0, 2, 2, 0, 2, 2, 2, 3]
    want = [0.4, None, 0.4, 0.4, None, 0.4, 0.4, 0.4, 0.0]
    for got, w in zip(margins, want):
        if w is None:
            assert np.isnan(got)
        else:
            assert got == pytest.approx(w, abs=1e-15)
    np.testing.assert_allclose(res.s, [10.0, 5.0, 1.0], rtol=0, atol=1e-14)


# ---------------------------------------------------------------- sign convention

def test_normalise_signs_hand_built_columns():
    """Sign rule of the output (the largest-magnitude entry of each U column is
    made positive, the first such entry on ties; V follows U): expected arrays
    written out by hand, including a negative maximum, a tie whose first entry
    is negative, a tie whose first entry is positive and a zero column."""
    u = np.array([[0.1, 0.5, -0.6, 0.4, 0.0],
                  [-0.9, 0.1, 0.6, -0.4, 0.0],
                  [0.3, -0.2, 0.1, 0.0, 0.0],
                  [0.2, 0.7, 0.0, 0.0, 0.0]])
    v = np.array([[1.0, 2.0, 3.0, 4.0, 5.0],
                  [-1.0, -2.0, -3.0, -4.0, -5.0]])
    s = np.array([5.0, 4.0, 3.0, 2.0, 0.0])
    un, sn, vn = H.normalise_signs(u, s, v)
    u_expect = np.array([[-0.1, 0.5, 0.6, 0.4, 0.0],
                         [0.9, 0.1, -0.6, -0.4, 0.0],
                         [-0.3, -0.2, -0.1, 0.0, 0.0],
                         [-0.2, 0.7, 0.0, 0.0, 0.0]])
    v_expect = np.array([[-1.0, 2.0, -3.0, 4.0, 5.0],
                         [1.0, -2.0, 3.0, -4.0, -5.0]])
    np.testing.assert_array_equal(un, u_expect)
    np.testing.assert_array_equal(vn, v_expect)
    np.testing.assert_array_equal(sn, s)


def test_sign_convention_worked_example():
    """A = [[0, -2], [3, 0], [0, 0]]: sigma = (3, 2); the rule fixes
    u1 = e2, v1 = e1 (A v1 = 3 u1) and u2 = e1, v2 = -e2 (A v2 = 2 u2), on
    every grid and in both tree orders."""
    a = np.array([[0.0, -2.0], [3.0, 0.0], [0.0, 0.0]])
    u_expect = np.array([[0.0, 1.0], [1.0, 0.0], [0.0, 0.0]])
    v_expect = np.array([[1.0, 0.0], [0.0, -1.0]])
    for br, bc in [(3, 2), (1, 1), (2, 1), (1, 2)]:
        for tree in ("col_then_row", "row_then_col"):
            res = H.hmat_svd(a, br, bc, Rule(H.FIXED_K, 2), tree=tree)
            np.testing.assert_allclose(res.s, [3.0, 2.0], rtol=1e-14)
            np.testing.assert_allclose(res.u, u_expect, atol=1e-14)
            np.testing.assert_allclose(res.v, v_expect, atol=1e-14)


def test_sign_convention_permuted_diagonal():
    """For a permuted diagonal matrix with entries of both signs every
    singular vector is a signed unit vector: the rule makes each u a +e_p and
    gives v the sign of the diagonal entry (A v = sigma u)."""
    g = np.random.default_rng(11)
    d = (np.arange(12, 0, -1, dtype=np.float64) + 0.5) * g.choice([-1.0, 1.0], 12)
    rows, cols = g.permutation(16)[:12], g.permutation(14)[:12]
    a = np.zeros((16, 14))
    a[rows, cols] = d
    for br, bc, tree in [(16, 14, "col_then_row"), (5, 4, "col_then_row"), (4, 5, "row_then_col")]:
        res = H.hmat_svd(a, br, bc, Rule(H.FIXED_K, 6), tree=tree)
        for i in range(6):
            u_e = np.zeros(16)
            u_e[rows[i]] = 1.0
            v_e = np.zeros(14)
            v_e[cols[i]] = np.sign(d[i])
            np.testing.assert_allclose(res.u[:, i], u_e, atol=1e-13)
            np.testing.assert_allclose(res.v[:, i], v_e, atol=1e-13)
