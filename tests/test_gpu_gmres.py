"""GMRES with the factor as right preconditioner (rsrs_gmres) against the oracle's GMRES with the
oracle's factor on the same inputs, and against the dense solution: same iteration counts (the
two factors agree to 1e-10), solutions to the tolerance, several right-hand sides at once,
restarts, the callback operator, an exact factor (one iteration) and the not-converged status."""
import numpy as np
import pytest

import workloads as W
from oracle import operators as ops
from oracle import refine as oref
from oracle import rsrs as orsrs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2311_01451_gb300 as pkg

    return pkg


def _to_gpu(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), device="cuda", dtype=torch.float64)


def _from_gpu(x):
    return x.cpu().numpy().T


CASES = {
    "grid2d_1024": lambda: W.small_problem(n_side=32, d=2, leaf=16, k=8, nrhs=3, seed_problem=1),
    "rand3d_1200": lambda: W.small_problem(n=1200, d=3, kernel="invr3d", leaf=20, k=8, nrhs=2, seed_problem=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_gmres_matches_oracle(R, name):
    pr = CASES[name]()
    tree_o, sched, fac, _ = orsrs.build(pr)
    op = ops.make_operator(pr)
    t = R.Tree(pr.points, pr.leaf)
    f = R.Factor(t, R.kind_of(pr.kernel), pr.k, fac.s, shift=pr.diag_shift, scale=pr.scale,
                 omega=pr.omega(fac.s), psi=pr.psi(fac.s))
    b = pr.rhs()
    X = torch.zeros_like(_to_gpu(b))
    rep = f.gmres(_to_gpu(b), X, rtol=1e-12, restart=20, maxit=40)
    assert rep.rel_residual <= 1e-12
    x = _from_gpu(X)
    xd = np.linalg.solve(op.dense(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    its = []
    for j in range(b.shape[1]):
        _, it, _ = oref.gmres(op.matvec, lambda v: orsrs.solve(fac, v), b[:, j], rtol=1e-12, restart=20)
        its.append(it)
    assert abs(rep.iterations - max(its)) <= 1
    # refinement with the same factor needs at least as many corrections
    Xr = torch.zeros_like(X)
    rr = f.refine(_to_gpu(b), Xr, rtol=1e-12, maxit=40)
    assert rep.iterations <= rr.iterations + 1


def test_gmres_mixed_and_restarts(R):
    pr = W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=4, seed_problem=3)
    tree = R.Tree(pr.points, pr.leaf)
    s = tree.info(pr.k).s_req_mixed
    f = R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                 precision=R.RSRS_PREC_MIXED, seed=5)
    b = pr.rhs()
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    for restart in (30, 2):
        X = torch.zeros_like(_to_gpu(b))
        rep = f.gmres(_to_gpu(b), X, rtol=1e-12, restart=restart, maxit=60)
        assert rep.rel_residual <= 1e-12
        assert np.linalg.norm(_from_gpu(X) - xd) / np.linalg.norm(xd) < 1e-11
        assert rep.history[0] == pytest.approx(1.0)
    # the not-converged status after too few iterations
    with pytest.raises(R.RSRSError) as e:
        f.gmres(_to_gpu(b), torch.zeros_like(_to_gpu(b)), rtol=1e-14, restart=30, maxit=1)
    assert e.value.name == "RSRS_E_NOT_CONVERGED"


def test_gmres_exact_factor_one_iteration(R):
    """A tree whose root is a leaf: the factor is the dense LU of A~ = Y pinv(Omega), exact to
    rounding, so A M^-1 = I and GMRES stops after one iteration."""
    pr = W.small_problem(n=400, d=2, leaf=512, k=8, nrhs=2, seed_problem=4)
    t = R.Tree(pr.points, pr.leaf)
    s = t.info(pr.k).s_req
    f = R.Factor(t, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale, seed=3)
    b = pr.rhs()
    X = torch.zeros_like(_to_gpu(b))
    rep = f.gmres(_to_gpu(b), X, rtol=1e-10, restart=10, maxit=10)
    assert rep.iterations == 1 and rep.rel_residual <= 1e-10


def test_gmres_callback_stencil(R):
    m = 12
    pr = W.Problem(name=f"stencil7_{m}cube", cfg=4, problem=0, d=3, kernel="stencil7",
                   points=W.grid_points_3d(m), leaf=27, k=8, s_cfg=0, nrhs=2, diag_shift=0.0, scale=1.0,
                   grid_side=m)
    st = R.Stencil7(pr.coefficients(), m)
    t = R.Tree(pr.points, pr.leaf)
    s = t.info(pr.k).s_req
    f = R.Factor(t, R.RSRS_OP_CALLBACK, pr.k, s, shift=0.0, scale=1.0, seed=7, matvec=st)
    b = pr.rhs()
    X = torch.zeros_like(_to_gpu(b))
    rep = f.gmres(_to_gpu(b), X, rtol=1e-12, restart=30, maxit=60)
    assert rep.rel_residual <= 1e-12
    r = b - ops.Stencil7Operator(m, pr.coefficients()).matvec(_from_gpu(X))
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-11
