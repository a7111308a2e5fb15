"""Pins of the oracle's GMRES (oracle.refine.gmres) by properties GMRES has in exact arithmetic:
finite termination in as many iterations as the minimal polynomial's degree (distinct eigenvalues
of a diagonalisable A M^-1), one iteration with the exact inverse as preconditioner, residual
estimates that never increase within a cycle and that equal the true residual, restarts that still
converge, and the solution of the dense system."""
import numpy as np
import pytest

from oracle import refine

pytestmark = pytest.mark.filterwarnings("ignore")


def _sym_with_eigs(eigs, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((len(eigs), len(eigs))))
    return q @ np.diag(eigs) @ q.T


@pytest.mark.parametrize("nd", [1, 2, 3, 5])
def test_terminates_after_distinct_eigenvalue_count(nd):
    eigs = np.repeat(np.arange(1, nd + 1, dtype=float), 40 // nd + 1)[:40]
    A = _sym_with_eigs(eigs, nd)
    b = np.random.default_rng(3).standard_normal(40)
    x, its, hist = refine.gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-12, restart=40, maxit=40)
    assert its == nd
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
    assert hist[-2] <= 1e-12 < hist[-3]  # the estimate reaches rtol at step nd, not before


def test_exact_preconditioner_one_iteration():
    A = np.random.default_rng(1).standard_normal((30, 30)) + 8 * np.eye(30)
    Ainv = np.linalg.inv(A)
    b = np.random.default_rng(2).standard_normal(30)
    x, its, hist = refine.gmres(lambda v: A @ v, lambda v: Ainv @ v, b, rtol=1e-12)
    assert its == 1
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_estimates_monotone_and_true_residual():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((60, 60)) / np.sqrt(60) + 2.5 * np.eye(60)  # nonsymmetric, well conditioned
    b = rng.standard_normal(60)
    x, its, hist = refine.gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-10, restart=60, maxit=60)
    est = hist[1:-1]
    assert all(a >= c * (1 - 1e-12) for a, c in zip(est, est[1:]))
    # the last estimate and the true residual agree to rounding
    assert abs(hist[-1] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) <= 1e-14
    assert hist[-1] <= 1e-10 and abs(est[-1] - hist[-1]) <= 1e-12


def test_restarts_converge_to_dense_solution():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((50, 50)) / np.sqrt(50) + 3.0 * np.eye(50)
    b = rng.standard_normal(50)
    x, its, hist = refine.gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-11, restart=4, maxit=200)
    assert hist[-1] <= 1e-11 and its > 4
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(x)


def test_preconditioned_matches_refinement_fixed_point():
    """With a good approximate inverse, GMRES needs no more iterations than refinement needs
    corrections (GMRES minimises the residual over the space refinement's iterates span)."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((80, 80)) / np.sqrt(80) + 4.0 * np.eye(80)
    Minv = np.linalg.inv(A + 1e-3 * rng.standard_normal((80, 80)))
    b = rng.standard_normal(80)
    x, its, hist = refine.gmres(lambda v: A @ v, lambda v: Minv @ v, b, rtol=1e-13)
    # refinement with the same approximate inverse
    xr = Minv @ b
    nref = 0
    while np.linalg.norm(b - A @ xr) > 1e-13 * np.linalg.norm(b):
        xr = xr + Minv @ (b - A @ xr)
        nref += 1
    assert its <= nref + 1
    assert np.linalg.norm(x - xr) <= 1e-11 * np.linalg.norm(x)
