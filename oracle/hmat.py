"""FP64 CPU oracle of the hierarchical merge-and-truncate (MAT) SVD.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path.

It follows the paper (Vasudevan & Ramakrishna, "A Hierarchical Singular
Value Decomposition Algorithm for Low Rank Matrices", arXiv:1710.02812)
step by step, each step written as its plain definition with LAPACK
(``numpy.linalg.svd``) as the only library primitive:

* block SVD of every block of the grid, truncated        -- Alg. 1 (DoSVDofColSlices)
* column merges over each row slab, binary tree           -- Section 3, column split; Alg. 1 (DoMergeOfSlices)
* slab step  V_j, Sigma_j = SVD(U_j^T X_j)                -- Section 3, Fig. 2; Alg. 1 (DoSVDofBlocks)
* row merges of the V_j Sigma_j, binary tree              -- Section 3, row split (Fig. 1); Alg. 1
* left-vector recovery  SVD(X V_r) = U_y S_y V_y^T,
  U = U_y, Sigma = S_y, V = V_r V_y                        -- Section 3, projection paragraph

Each merge is the plain MAT: the exact SVD of the concatenation
[U1 S1 | U2 S2], then truncation (Section 3, column split).  The paper's
faster orthogonal-complement form (Section 3, Eqs. orthmerge1/orthmerge,
after Brand) reaches the same result; ``mat_merge_orth`` implements it as a
checked alternative.

Readings of points where the paper is silent, garbled or ambiguous:

1. Eq. orthmerge1 prints the lower-right block of E as Sigma_2 R.  Since
   U2 S2 = U1 P S2 + U_o R S2 with P = U1^T U2, the block is R Sigma_2.
2. Q = U2 - U1 U1^T U2 may be rank deficient (sibling blocks of a low-rank
   matrix share their column space).  ``mat_merge_orth`` takes U_o from an
   SVD of Q and keeps only the directions above rounding level, so E has
   k + r' rows (r' <= l) and k + l columns.
3. Truncation "up to gamma sigma_1" keeps sigma_i >= gamma * sigma_1, with
   sigma_1 the largest singular value of that block or merged result.
   Fixed-k keeps min(k, numerical rank).  Energy keeps the smallest r with
   sum_{i<=r} sigma_i^2 >= f * total, where total is the energy of what is
   being truncated (||B||_F^2 for a block, ||S1||^2 + ||S2||^2 for a merge).
   Every rule also drops sigma_i <= rank_tol * sigma_1 (numerically zero)
   and caps the rank at rank_cap.
4. The slab SVD (Alg. 1, DoSVDofBlocks) is truncated by the same rule.
5. N_d = round(m/d + 0.5) is read as ceil(m/d); the last slab/slice is
   smaller (ragged).
6. DoMergeOfSlices: merge adjacent pairs (0,1),(2,3),...; an odd last
   element is carried unchanged to the next level; repeat until one element
   remains (ceil(log2 N) levels); return it.
7. "V_r is an r x m orthogonal matrix" means n x r with orthonormal columns.
8. Signs of singular vectors are not unique; results are normalised so the
   largest-magnitude entry of each U column is positive (V follows).
9. Alg. 2 (iterative improvement) measures Error = ||Sigma_hat - Sigma_tilde||_2
   / ||Sigma_hat||_2 of diagonal matrices: the spectral norm, i.e. the largest
   |sigma_hat_i - sigma_tilde_i| over sigma_hat_1 (a value missing from one of
   the two lists counts as zero).
10. Alg. 2 as printed never updates V_hat inside its loop, so every pass would
   repeat the same computation; read as V_hat <- V_tilde after each pass (the
   power-iteration reading the paper gives for the algorithm).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import numpy as np

FIXED_K = "fixed_k"
GAMMA = "gamma"
ENERGY = "energy"


@dataclass
class Rule:
    """Truncation rule applied after every SVD of the path (Section 3, MAT).

    mode: ``fixed_k`` (param = k), ``gamma`` (param = gamma), or ``energy``
    (param = kept energy fraction f).  ``rank_cap`` bounds every rank;
    ``rank_tol`` is the relative level below which a singular value counts
    as zero.
    """

    mode: str = FIXED_K
    param: float = 10
    rank_cap: int = 256
    rank_tol: float = 1e-12

    def rank(self, sigma: np.ndarray, total: Optional[float] = None) -> int:
        """Number of singular values kept (Section 3: truncation before and
        after every merge; reading 3 of the module docstring)."""
        sigma = np.asarray(sigma, dtype=np.float64)
        if sigma.size == 0 or not sigma[0] > 0.0:
            return 0
        numerical = int(np.count_nonzero(sigma > self.rank_tol * sigma[0]))
        if self.mode == FIXED_K:
            r = int(self.param)
        elif self.mode == GAMMA:
            r = int(np.count_nonzero(sigma >= self.param * sigma[0]))
        elif self.mode == ENERGY:
            if total is None:
                total = float(np.sum(sigma * sigma))
            cum = np.cumsum(sigma * sigma)
            hit = np.nonzero(cum >= self.param * total)[0]
            r = int(hit[0]) + 1 if hit.size else int(sigma.size)
        else:
            raise ValueError(f"unknown truncation mode {self.mode!r}")
        return max(0, min(r, numerical, self.rank_cap, sigma.size))


@dataclass
class Trace:
    """Rank decisions and the margin of the deciding value, per step."""

    steps: List[Tuple[str, int, float]] = field(default_factory=list)

    def add(self, name: str, sigma: np.ndarray, r: int, rule: Rule):
        margin = float("nan")
        if sigma.size and sigma[0] > 0 and rule.mode == GAMMA:
            thr = rule.param * sigma[0]
            margin = float(np.min(np.abs(sigma - thr)) / sigma[0])
        self.steps.append((name, r, margin))


def thin_svd(a: np.ndarray):
    """Exact thin SVD (LAPACK through numpy), singular values descending."""
    if a.shape[0] == 0 or a.shape[1] == 0:
        kk = min(a.shape)
        return (np.zeros((a.shape[0], kk)), np.zeros(kk), np.zeros((a.shape[1], kk)))
    u, s, vt = np.linalg.svd(a, full_matrices=False)
    return u, s, vt.T


def block_svd(b: np.ndarray, rule: Rule, trace: Optional[Trace] = None, name="block"):
    """Truncated SVD of one block: U_B, Sigma_B (Alg. 1, DoSVDofColSlices;
    the block's V is not propagated, Section 3 column split)."""
    b = np.asarray(b, dtype=np.float64)
    u, s, _ = thin_svd(b)
    r = rule.rank(s, total=float(np.sum(b * b)))
    if trace is not None:
        trace.add(name, s, r, rule)
    return u[:, :r].copy(), s[:r].copy()


def mat_merge(u1, s1, u2, s2, rule: Rule, trace: Optional[Trace] = None, name="merge"):
    """Plain MAT merge (Section 3, column split):
    [X1 X2] ~ [U1 S1 | U2 S2] blkdiag(V1, V2)^T; the SVD of the
    concatenation gives U and Sigma, which are then truncated."""
    c = np.concatenate([u1 * s1[None, :], u2 * s2[None, :]], axis=1)
    u, s, _ = thin_svd(c)
    total = float(np.sum(s1 * s1) + np.sum(s2 * s2))
    r = rule.rank(s, total=total)
    if trace is not None:
        trace.add(name, s, r, rule)
    return u[:, :r].copy(), s[:r].copy()


def mat_merge_orth(u1, s1, u2, s2, rule: Rule, return_core: bool = False):
    """Orthogonal-complement merge (Section 3, Eqs. orthmerge1 and
    orthmerge, after Brand):  P = U1^T U2,  Q = U2 - U1 P = U_o R,
    E = [[S1, P S2], [0, R S2]],  E = U_E S_E V_E^T,  U = [U1 U_o] U_E.
    Reading 1 (R S2, not S2 R) and reading 2 (rank-deficient Q)."""
    k1 = s1.shape[0]
    l = s2.shape[0]
    h = u1.shape[0]
    p = u1.T @ u2
    q = u2 - u1 @ p
    # U_o, R from an SVD of Q: Q = Uq Sq Vq^T, take U_o = Uq, R = Sq Vq^T on
    # the directions that are not at rounding level (reading 2).
    uq, sq, vq = thin_svd(q)
    keep = sq > max(h, l, 1) * np.finfo(np.float64).eps
    uo = uq[:, keep]
    rr = (sq[keep, None] * vq[:, keep].T)
    rp = uo.shape[1]
    e = np.zeros((k1 + rp, k1 + l))
    e[:k1, :k1] = np.diag(s1)
    e[:k1, k1:] = p * s2[None, :]
    e[k1:, k1:] = rr * s2[None, :]
    ue, se, _ = thin_svd(e)
    total = float(np.sum(s1 * s1) + np.sum(s2 * s2))
    r = rule.rank(se, total=total)
    u = np.concatenate([u1, uo], axis=1) @ ue[:, :r]
    if return_core:
        return u, se[:r].copy(), e
    return u, se[:r].copy()


def merge_tree(items: list, merge: Callable):
    """DoMergeOfSlices (Alg. 1) under reading 6: pair adjacent elements,
    carry an odd last element, repeat until one remains.  ``items`` is a
    list of (U, Sigma); ``merge(a, b, level, index)`` merges two of them."""
    if not items:
        raise ValueError("merge_tree needs at least one element")
    level = 0
    while len(items) > 1:
        nxt = []
        for i in range(0, len(items) - 1, 2):
            nxt.append(merge(items[i], items[i + 1], level, i // 2))
        if len(items) % 2:
            nxt.append(items[-1])
        items = nxt
        level += 1
    return items[0]


def tree_schedule(count: int) -> List[List[Tuple[int, int]]]:
    """The pairs merged at each level of DoMergeOfSlices (reading 6), as
    positions in that level's list; an odd last element is carried."""
    levels = []
    while count > 1:
        levels.append([(i, i + 1) for i in range(0, count - 1, 2)])
        count = (count + 1) // 2
    return levels


def grid(m: int, n: int, block_rows: int, block_cols: int):
    """Row-slab and column-slice boundaries (Alg. 1, reading 5: ceil)."""
    rows = [(r0, min(r0 + block_rows, m)) for r0 in range(0, m, block_rows)]
    cols = [(c0, min(c0 + block_cols, n)) for c0 in range(0, n, block_cols)]
    return rows, cols


def slab_step(u_j, x_j, rule: Rule, trace: Optional[Trace] = None, name="slab"):
    """V_j, Sigma_j = SVD(U_j^T X_j) (Section 3, Fig. 2; Alg. 1
    DoSVDofBlocks), truncated by the same rule (reading 4).  Returns the
    right singular vectors V_j (n x r) and Sigma_j."""
    z = u_j.T @ np.asarray(x_j, dtype=np.float64)
    _, s, v = thin_svd(z)
    r = rule.rank(s)
    if trace is not None:
        trace.add(name, s, r, rule)
    return v[:, :r].copy(), s[:r].copy()


def recover_left(x, v_r):
    """Left-vector recovery by projection (Section 3): Y = X V_r =
    U_y S_y V_y^T gives U = U_y, Sigma = S_y, V = V_r V_y, the exact SVD of
    X V_r V_r^T."""
    y = np.asarray(x, dtype=np.float64) @ v_r
    uy, sy, vy = thin_svd(y)
    return uy, sy, v_r @ vy


def normalise_signs(u, s, v):
    """Make the largest-magnitude entry of each U column positive."""
    if u.shape[1] == 0:
        return u, s, v
    idx = np.argmax(np.abs(u), axis=0)
    sg = np.sign(u[idx, np.arange(u.shape[1])])
    sg[sg == 0] = 1.0
    return u * sg[None, :], s, v * sg[None, :]


@dataclass
class Result:
    u: np.ndarray
    s: np.ndarray
    v: np.ndarray
    trace: Trace
    v_hat: np.ndarray
    s_hat: np.ndarray


def hmat_svd(x, block_rows: int, block_cols: int, rule: Rule,
             tree: str = "col_then_row", merge: str = "plain") -> Result:
    """The whole path of Alg. 1 plus the projection step of Section 3.

    ``tree='col_then_row'`` is the paper's order: column MAT inside each row
    slab, slab step, row MAT over the slabs, then left-vector recovery.
    ``tree='row_then_col'`` runs the same algorithm on X^T and swaps U, V.
    ``merge='orth'`` uses the orthogonal-complement merge instead of the
    plain concatenated SVD (they agree; see ``mat_merge_orth``)."""
    x = np.asarray(x)
    if tree == "row_then_col":
        res = hmat_svd(x.T, block_cols, block_rows, rule, "col_then_row", merge)
        u, s, v = normalise_signs(res.v, res.s, res.u)
        return Result(u, s, v, res.trace, res.v_hat, res.s_hat)
    if tree != "col_then_row":
        raise ValueError(f"unknown tree {tree!r}")
    m, n = x.shape
    if m < 1 or n < 1 or block_rows < 1 or block_cols < 1:
        raise ValueError("empty matrix or block")
    trace = Trace()
    rows, cols = grid(m, n, block_rows, block_cols)

    def do_merge(a, b, level, idx, tag):
        fn = mat_merge if merge == "plain" else mat_merge_orth
        if fn is mat_merge:
            return mat_merge(a[0], a[1], b[0], b[1], rule, trace, f"{tag}L{level}#{idx}")
        u, s = mat_merge_orth(a[0], a[1], b[0], b[1], rule)
        return u, s

    slabs = []
    for j, (r0, r1) in enumerate(rows):
        xj = np.asarray(x[r0:r1], dtype=np.float64)
        leaves = [block_svd(xj[:, c0:c1], rule, trace, f"block{j},{c}")
                  for c, (c0, c1) in enumerate(cols)]
        u_j, _ = merge_tree(leaves, lambda a, b, lv, i: do_merge(a, b, lv, i, f"col{j}"))
        slabs.append(slab_step(u_j, xj, rule, trace, f"slab{j}"))
    v_hat, s_hat = merge_tree(slabs, lambda a, b, lv, i: do_merge(a, b, lv, i, "row"))
    u, s, v = recover_left(x, v_hat)
    u, s, v = normalise_signs(u, s, v)
    return Result(u, s, v, trace, v_hat, s_hat)


def truncated_svd(x, r: int):
    """Full SVD followed by truncation to rank r: the paper's comparator
    X_k (Section 4)."""
    u, s, v = thin_svd(np.asarray(x, dtype=np.float64))
    return normalise_signs(u[:, :r], s[:r], v[:, :r])


def relative_error(x_k: np.ndarray, xhat_k: np.ndarray) -> float:
    """||X_k - Xhat_k||_F / ||X_k||_F, the paper's error measure (Section 4)."""
    den = np.linalg.norm(x_k)
    return float(np.linalg.norm(x_k - xhat_k) / den) if den > 0 else 0.0


@dataclass
class Refined:
    u: np.ndarray
    s: np.ndarray
    v: np.ndarray
    errors: List[float]

    @property
    def iterations(self) -> int:
        return len(self.errors)


def iterative_improvement(x, v_hat, s_hat, eps: float = 1e-3, max_iters: int = 50,
                          rank_tol: float = 0.0) -> Refined:
    """Alg. 2 (iterative improvement), readings 9 and 10: repeat
    Ũ_i, Σ̃_i, Ṽ_i^T = SVD(X V̂);  Ũ, Σ̃, Ṽ^T = SVD(Ũ_i^T X);
    Error = max_i |σ̂_i - σ̃_i| / σ̂_1;  Σ̂ = Σ̃;  V̂ = Ṽ
    while Error > eps (at most max_iters passes); return Û = Ũ_i Ũ, Σ̂, V̂.
    Singular values at or below rank_tol * σ_1 of a pass are dropped (with
    their vectors), as every truncation on the path does."""
    x = np.asarray(x, dtype=np.float64)
    v_hat = np.asarray(v_hat, dtype=np.float64)
    s_hat = np.asarray(s_hat, dtype=np.float64)
    errors: List[float] = []
    u_hat = np.zeros((x.shape[0], 0))

    def keep(u, s, v):
        r = int(np.sum(s > rank_tol * s[0])) if s.size and s[0] > 0 else 0
        return u[:, :r], s[:r], v[:, :r]

    for _ in range(max(1, max_iters)):
        ui, si, _ = keep(*thin_svd(x @ v_hat))
        ut, st, vt = keep(*thin_svd(ui.T @ x))
        r = max(s_hat.size, st.size)
        a = np.zeros(r)
        b = np.zeros(r)
        a[:s_hat.size] = s_hat
        b[:st.size] = st
        err = float(np.max(np.abs(a - b)) / s_hat[0]) if s_hat.size and s_hat[0] > 0 else 0.0
        errors.append(err)
        u_hat, s_hat, v_hat = ui @ ut, st, vt
        if err <= eps:
            break
    u_hat, s_hat, v_hat = normalise_signs(u_hat, s_hat, v_hat)
    return Refined(u_hat, s_hat, v_hat, errors)
