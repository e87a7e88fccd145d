"""Pins for the oracle's comparison measures (the parity tests' pass/fail).

A measure that always returned 0 would make every parity test pass, so each
is checked here against values fixed by hand: planted rotations by a known
angle, rotations inside a cluster of equal singular values (which must not
count), gap splits and relative errors worked out from the definitions.
"""
import numpy as np
import pytest

import oracle
from oracle import metrics as Mx


def _e(n, *idx):
    """Columns of the n x n identity."""
    return np.eye(n)[:, list(idx)]


@pytest.mark.parametrize("theta", [1e-7, 1e-3, 0.3, 1.2, np.pi / 2])
def test_principal_angle_of_a_planted_rotation(theta):
    a = _e(5, 0, 1)
    b = a.copy()
    b[:, 1] = np.cos(theta) * _e(5, 1)[:, 0] + np.sin(theta) * _e(5, 3)[:, 0]
    assert oracle.principal_angle(a, b) == pytest.approx(theta, rel=1e-9, abs=1e-15)
    assert oracle.principal_angle(b, a) == pytest.approx(theta, rel=1e-9, abs=1e-15)


def test_principal_angle_ignores_bases_and_signs():
    rng = np.random.default_rng(3)
    a, _ = np.linalg.qr(rng.standard_normal((9, 3)))
    r, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    assert oracle.principal_angle(a, a @ r) < 1e-14
    assert oracle.principal_angle(a, -a) < 1e-14
    # a different 3-dimensional subspace is detected, and unequal sizes are orthogonal
    b, _ = np.linalg.qr(rng.standard_normal((9, 3)))
    assert oracle.principal_angle(a, b) > 0.1
    assert oracle.principal_angle(a, a[:, :2]) == pytest.approx(np.pi / 2)


def test_sigma_rel_err_worked_values():
    ref = [4.0, 2.0, 1.0]
    test = [4.004, 2.0, 0.9]
    assert oracle.sigma_rel_err(test, ref) == pytest.approx(0.1, rel=1e-12)
    assert oracle.sigma_rel_err(test, ref, 2) == pytest.approx(1e-3, rel=1e-9)
    assert oracle.sigma_rel_err(test, ref, 0) == 0.0
    # relative to the reference value, not the tested one
    assert oracle.sigma_rel_err([2.0], [1.0]) == pytest.approx(1.0)
    assert oracle.sigma_rel_err([1.0], [2.0]) == pytest.approx(0.5)


def test_gap_groups_worked_split():
    s = [10.0, 9.95, 5.0, 4.99, 4.98, 1.0]
    # 10 -> 9.95 differs by 0.5% (< 1%): one group; 9.95 -> 5 splits; 5, 4.99, 4.98
    # stay together; 4.98 -> 1 splits
    assert Mx.gap_groups(s, 1e-2) == [(0, 2), (2, 5), (5, 6)]
    assert Mx.gap_groups(s, 1e-3) == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    assert Mx.gap_groups([], 1e-2) == []


def test_gap_prefix_worked_values():
    s = [10.0, 9.95, 5.0, 4.99, 1.0]
    assert oracle.gap_prefix(s, 1) == 0      # 10 and 9.95 are not separated
    assert oracle.gap_prefix(s, 2) == 2
    assert oracle.gap_prefix(s, 3) == 2      # 5 and 4.99 are not separated
    assert oracle.gap_prefix(s, 4) == 4
    assert oracle.gap_prefix(s, 5) == 5      # the end of the list counts as a gap
    assert oracle.gap_prefix(s, 9) == 5


def test_leading_subspace_angle_counts_tilts_but_not_cluster_rotations():
    n = 7
    u_ref = _e(n, 0, 1, 2, 3)
    s_ref = [3.0, 2.0, 2.0, 1.0]            # columns 1 and 2 form a cluster
    c, s = np.cos(0.4), np.sin(0.4)
    rot = u_ref.copy()
    rot[:, 1], rot[:, 2] = c * u_ref[:, 1] - s * u_ref[:, 2], s * u_ref[:, 1] + c * u_ref[:, 2]
    assert oracle.leading_subspace_angle(rot, u_ref, s_ref) < 1e-14
    assert Mx.subspace_angles_grouped(rot, u_ref, s_ref) < 1e-14
    theta = 0.05
    tilt = u_ref.copy()
    tilt[:, 1] = np.cos(theta) * u_ref[:, 1] + np.sin(theta) * _e(n, 5)[:, 0]
    assert oracle.leading_subspace_angle(tilt, u_ref, s_ref) == pytest.approx(theta, rel=1e-9)
    assert Mx.subspace_angles_grouped(tilt, u_ref, s_ref) == pytest.approx(theta, rel=1e-9)
    # up to 2 columns the cluster is cut: only the first column is determined
    assert oracle.leading_subspace_angle(tilt, u_ref, s_ref, upto=2) < 1e-14
    # a swap of the leading and the last direction is a right angle
    swap = u_ref[:, [3, 1, 2, 0]]
    assert Mx.subspace_angles_grouped(swap, u_ref, s_ref) == pytest.approx(np.pi / 2)
    assert oracle.leading_subspace_angle(swap, u_ref, s_ref, upto=1) == pytest.approx(np.pi / 2)


def test_orthonormality_defect_worked_value():
    u = _e(3, 0, 1)
    assert Mx.orthonormality_defect(u) == 0.0
    u[:, 1] *= 1.001
    assert Mx.orthonormality_defect(u) == pytest.approx(1.001 ** 2 - 1, rel=1e-12)
    v = _e(3, 0, 1)
    v[2, 0] = 0.01                           # (e0 + 0.01 e2) . e1 = 0; norm^2 - 1 = 1e-4
    assert Mx.orthonormality_defect(v) == pytest.approx(1e-4, rel=1e-9)
