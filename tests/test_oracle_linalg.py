"""Pins for the oracle's null space, pseudoinverse, CPQR-based ID and operators (Sec. 2, Sec. 5)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import linalg as la
from oracle import operators as ops


def test_null_basis():
    rng = np.random.default_rng(1)
    m = rng.standard_normal((37, 60))
    n = la.null(m)
    assert n.shape == (60, 23)
    assert np.abs(m @ n).max() < 1e-13
    assert np.abs(n.T @ n - np.eye(23)).max() < 1e-14


def test_pinv_right_matches_svd_pinv():
    rng = np.random.default_rng(2)
    m = rng.standard_normal((30, 55))
    y = rng.standard_normal((7, 55))
    assert np.allclose(la.pinv_right(y, m), y @ np.linalg.pinv(m), rtol=0, atol=1e-13)
    # block extraction (eq. pinvformula): Y = X M with exact X is recovered
    x = rng.standard_normal((7, 30))
    assert np.abs(la.pinv_right(x @ m, m) - x).max() < 1e-12


def test_cpqr_matches_lapack_pivoted_qr():
    rng = np.random.default_rng(3)
    # a matrix with decaying singular values, rows = box points
    u, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    v, _ = np.linalg.qr(rng.standard_normal((300, 40)))
    m = (u * np.logspace(0, -12, 40)) @ v.T  # 40 x 300
    k = 15
    skel, red, t = la.cpqr_id(m, k, tau=1e-14)
    _, r, piv = sla.qr(m.T, mode="economic", pivoting=True)
    assert np.array_equal(skel, piv[:k])
    t_ref = sla.solve_triangular(r[:k, :k], r[:k, k:])
    order = np.argsort(piv[k:])
    assert np.allclose(t, t_ref[:, order], rtol=0, atol=1e-10 * max(1, np.abs(t_ref).max()))
    assert np.array_equal(red, np.sort(piv[k:]))
    # ID identity: ||M_red - T^T M_skel||_F = ||R22||_F
    resid = np.linalg.norm(m[red] - t.T @ m[skel])
    assert abs(resid - np.linalg.norm(np.triu(r[k:, k:]))) <= 1e-9 * resid + 1e-15
    # near-optimality (Sec. 2.3): error within a modest factor of sigma_{k+1}
    sig = np.linalg.svd(m, compute_uv=False)
    assert resid <= math.sqrt(1 + k * (40 - k)) * 10 * sig[k]


def test_cpqr_exact_low_rank_truncation():
    rng = np.random.default_rng(4)
    m = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 80))  # rank 4
    skel, red, t = la.cpqr_id(m, 8, tau=64 * np.finfo(float).eps * 80)
    assert len(skel) == 8 and len(red) == 22
    # dependent pivots (5..8) get zero interpolation rows; the ID is exact to rounding
    assert np.abs(t[4:]).max() == 0.0
    assert np.abs(t).max() < 1e3
    assert np.linalg.norm(m[red] - t.T @ m[skel]) < 1e-12 * np.linalg.norm(m)


def test_cpqr_tie_goes_to_lowest_index():
    m = np.zeros((3, 5))
    m[0, 0] = m[2, 1] = 1.0  # rows 0 and 2 have equal norm
    m[1, 2] = 0.5
    skel, red, _ = la.cpqr_id(m, 1, tau=1e-14)
    assert skel[0] == 0


def test_kernel_entries_scalar_formula():
    pts2 = W.uniform_points(50, 2, W.rng_for(95, 0, 0))
    pts3 = W.uniform_points(50, 3, W.rng_for(95, 1, 0))
    idx = np.arange(50)
    k2 = ops.kernel_entries("log2d", pts2, pts2, idx, idx)
    k3 = ops.kernel_entries("invr3d", pts3, pts3, idx, idx)
    for i, j in [(0, 1), (3, 7), (49, 2), (10, 10)]:
        e2 = 0.0 if i == j else math.log(math.dist(pts2[i], pts2[j]))
        e3 = 0.0 if i == j else 1.0 / math.dist(pts3[i], pts3[j])
        assert abs(k2[i, j] - e2) <= 1e-15 * max(1, abs(e2))
        assert abs(k3[i, j] - e3) <= 1e-14 * max(1, abs(e3))


def test_kernel_operator_is_symmetric_and_samples_match_dense():
    pr = W.small_problem(n=300, d=2)
    op = ops.make_operator(pr)
    a = op.dense()
    assert np.array_equal(a, a.T)
    assert np.all(np.diag(a) == 1.0)
    x = np.random.default_rng(5).standard_normal((300, 3))
    assert np.abs(op.matvec(x) - a @ x).max() < 1e-13


def test_stencil7_closed_forms():
    m = 6
    op = ops.Stencil7Operator(m, np.ones(m ** 3))
    a = op.dense()
    assert np.allclose(a, a.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(a).min() > 0
    # constant coefficient: A 1 counts boundary faces (beta = 2 on each), interior rows sum to 0
    g = np.arange(m)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    nb = sum(((c == 0).astype(int) + (c == m - 1).astype(int)) for c in (x, y, z)).ravel()
    assert np.allclose(a @ np.ones(m ** 3), 2.0 * nb)
    # two cells with different coefficients: harmonic-mean face
    coef = np.ones(m ** 3)
    coef[0], coef[1] = 1.0, 3.0
    a2 = ops.Stencil7Operator(m, coef).dense()
    assert math.isclose(-a2[0, 1], 2 * 1.0 * 3.0 / 4.0)


def test_cpqr_rows_below_the_absolute_floor_are_dependent():
    """A sketch at the rounding level of what was cancelled (floor): every pivot is dependent, the
    skeletons are the first k rows in original order and T = 0."""
    rng = np.random.default_rng(11)
    m = 1e-17 * rng.standard_normal((12, 40))
    skel, red, t = la.cpqr_id(m, 5, 1e-10, floor=1e-10)
    assert list(skel) == [0, 1, 2, 3, 4] and list(red) == list(range(5, 12))
    assert not t.any()
    # without the floor the same matrix is ranked by its noise
    skel2, _, t2 = la.cpqr_id(m, 5, 1e-10)
    assert list(skel2) != [0, 1, 2, 3, 4] and t2.any()
