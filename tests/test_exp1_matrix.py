"""The matrix of the paper's Experiment 1 (Sec. 5.1): its diagonal, the cell integral of the log
kernel, in closed form against 2D adaptive quadrature (the paper uses Quadpack for it), and the
sample count the tree gives for it against the paper's n_samples."""
import numpy as np
import pytest

import workloads as W

integrate = pytest.importorskip("scipy.integrate")


@pytest.mark.parametrize("h", [1.0, 1.0 / 284, 0.37, 1.0 / 1132])
def test_cell_log_mean_matches_quadrature(h):
    a = h / 2
    # [-a, a]^2 is 8 copies of the triangle 0 <= y <= x <= a (log singular only at the corner)
    tri, _ = integrate.dblquad(lambda y, x: 0.5 * np.log(x * x + y * y), 0, a, 0, lambda x: x,
                               epsabs=1e-15, epsrel=1e-13)
    assert W.cell_log_mean(h) == pytest.approx(8 * tri / h ** 2, rel=1e-12, abs=1e-13)


def test_exp1_operator_entries():
    pr = W.exp1_problem(n_side=16, k=8)
    from oracle import operators as ops
    A = ops.make_operator(pr).dense()
    n = pr.n
    i, j = 3, 200
    r = np.linalg.norm(pr.points[i] - pr.points[j])
    assert A[i, j] == pytest.approx(np.log(r) / n, rel=1e-14)
    assert A[5, 5] == pytest.approx(W.cell_log_mean(1 / 16) / n, rel=1e-14)
    assert pr.leaf == 32


def test_exp1_sample_count_is_the_papers():
    lib = pytest.importorskip("paper_2311_01451_gb300")
    pr = W.exp1_problem()
    assert pr.n == 80656
    t = lib.Tree(pr.points, pr.leaf)
    assert t.info(pr.k).s_req == 1520  # n_samples of the paper's Exp. 1 table for k = 40
