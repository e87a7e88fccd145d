"""Comparison measures used by the parity tests (TEST INFRASTRUCTURE ONLY).

Singular vectors are unique only up to sign, and only up to rotation inside
a cluster of equal singular values, so subspaces are compared through
principal angles over groups separated by a relative gap; singular values are
compared directly.
"""
from __future__ import annotations

import numpy as np


def sigma_rel_err(s_test, s_ref, k=None):
    """max_i |s_test_i - s_ref_i| / s_ref_i over the first k values."""
    s_test = np.asarray(s_test, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    k = min(s_test.size, s_ref.size) if k is None else k
    if k == 0:
        return 0.0
    return float(np.max(np.abs(s_test[:k] - s_ref[:k]) / s_ref[:k]))


def principal_angle(a, b) -> float:
    """Largest principal angle (radians) between span(a) and span(b), both
    with orthonormal columns: asin of ||(I - a a^T) b||_2, symmetrised."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape[1] == 0 and b.shape[1] == 0:
        return 0.0
    if a.shape[1] != b.shape[1]:
        return float(np.pi / 2)
    res = b - a @ (a.T @ b)
    sv = np.linalg.norm(res, 2)
    res2 = a - b @ (b.T @ a)
    sv = max(sv, np.linalg.norm(res2, 2))
    return float(np.arcsin(min(1.0, sv)))


def gap_groups(s, rel_gap=1e-2):
    """Split indices 0..len(s)-1 into runs whose neighbouring values differ
    by less than rel_gap (relative to the larger one)."""
    s = np.asarray(s, dtype=np.float64)
    groups, start = [], 0
    for i in range(1, s.size):
        if (s[i - 1] - s[i]) > rel_gap * s[i - 1]:
            groups.append((start, i))
            start = i
    if s.size:
        groups.append((start, s.size))
    return groups


def subspace_angles_grouped(u_test, u_ref, s_ref, rel_gap=1e-2, upto=None):
    """Largest principal angle over the leading gap-separated groups.

    Groups are formed on s_ref; a group is compared only if it is separated
    from the next value by rel_gap.  ``upto`` limits the comparison to the
    first ``upto`` columns (rounded down to a group boundary)."""
    s_ref = np.asarray(s_ref, dtype=np.float64)
    upto = s_ref.size if upto is None else min(upto, s_ref.size)
    worst = 0.0
    for g0, g1 in gap_groups(s_ref[:upto], rel_gap):
        if g1 >= upto and upto < s_ref.size:
            # last group must be separated from what follows
            if not (s_ref[g1 - 1] - s_ref[g1]) > rel_gap * s_ref[g1 - 1]:
                break
        worst = max(worst, principal_angle(u_test[:, g0:g1], u_ref[:, g0:g1]))
    return worst


def leading_subspace_angle(u_test, u_ref, s_ref, rel_gap=1e-2, upto=None):
    """Angle between the spans of the first j columns, where j is the
    largest index <= upto with a relative gap after it."""
    s_ref = np.asarray(s_ref, dtype=np.float64)
    upto = s_ref.size if upto is None else min(upto, s_ref.size)
    j = 0
    for i in range(1, upto + 1):
        if i == s_ref.size or (s_ref[i - 1] - s_ref[i]) > rel_gap * s_ref[i - 1]:
            j = i
    if j == 0:
        return 0.0
    return principal_angle(u_test[:, :j], u_ref[:, :j])


def orthonormality_defect(u) -> float:
    u = np.asarray(u, dtype=np.float64)
    if u.shape[1] == 0:
        return 0.0
    return float(np.max(np.abs(u.T @ u - np.eye(u.shape[1]))))


def gap_prefix(s_true, k, rel_gap=1e-2):
    """Largest j <= k such that s_true[j-1] is separated from s_true[j] by a
    relative gap (j == len(s_true) counts as separated).  Singular values and
    subspaces beyond such a gap, inside a dense cluster, are not determined
    to better than the cluster width and are not gated."""
    s_true = np.asarray(s_true, dtype=np.float64)
    best = 0
    for j in range(1, min(k, s_true.size) + 1):
        if j == s_true.size or (s_true[j - 1] - s_true[j]) > rel_gap * s_true[j - 1]:
            best = j
    return best
