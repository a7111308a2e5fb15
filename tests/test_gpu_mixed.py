"""Mixed-precision variants against each other and against the FP64 oracle after refinement.

The mixed path's CPQR runs its reflectors in FP32 on the sketch held in distributed shared memory
(pivots on FP64 norm sums) or, on request, in FP64 in global memory.  The projected sketch it
factors already carries FP32 rounding, so the two may differ on pivots whose residuals are within
FP32 resolution of each other; both factors must precondition equally well and refine to the FP64
oracle's solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as ops

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


def _to_gpu(b):
    return torch.tensor(np.ascontiguousarray(np.asarray(b).T), device="cuda", dtype=torch.float64)


CASES = {
    "grid2d_4096": lambda: W.config(0)[0],
    "rand2d_3000": lambda: W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=2, seed_problem=3),
    "rand3d_1500": lambda: W.small_problem(n=1500, d=3, kernel="invr3d", leaf=20, k=8, nrhs=2, seed_problem=4),
    # leaves of up to 340 points: colour groups whose X_RR blocks exceed 224 rows take the FP64 LU
    # route to X_RR^-1, the others the FP32 Gauss-Jordan one, in the same factor
    "rand2d_bigleaf_4000": lambda: W.small_problem(n=4000, d=2, leaf=340, k=10, nrhs=2, seed_problem=6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_cpqr_variants(R, name):
    pr = CASES[name]()
    tree = R.Tree(pr.points, pr.leaf)
    s = max(pr.s_cfg, tree.info(pr.k).s_req_mixed)
    b = pr.rhs()
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    fac, its = {}, {}
    for mc in (0, 1):
        f = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                     precision=R.RSRS_PREC_MIXED, seed=21, mixed_cpqr=mc)
        X = torch.zeros_like(_to_gpu(b))
        rep = f.refine(_to_gpu(b), X, rtol=1e-13, maxit=40)
        assert rep.rel_residual <= 1e-13
        assert rep.history[0] < 1e-2, (mc, rep.history[0])
        x = X.cpu().numpy().T
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-11
        fac[mc] = f
        its[mc] = rep.iterations
    # the two factors precondition alike (on grids, FP32 rounding breaks the many exact pivot ties
    # differently, so skeleton lists are not compared)
    assert abs(its[0] - its[1]) <= 1
    assert fac[0].stats().n_boxes == fac[1].stats().n_boxes


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_tensor_core_products(R, name):
    """Grams, their blocked Cholesky factors and L^-T, least-squares right-hand sides, projection
    solves and updates as 3xTF32 tcgen05 products (default) against the FP32 SIMT kernels
    (substitution with the Cholesky factor): both factors precondition alike and refine to the
    dense solution."""
    pr = CASES[name]()
    tree = R.Tree(pr.points, pr.leaf)
    s = max(pr.s_cfg, tree.info(pr.k).s_req_mixed)
    b = pr.rhs()
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    its = {}
    for mg in (0, 1):
        f = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                     precision=R.RSRS_PREC_MIXED, seed=22, mixed_gemm=mg)
        X = torch.zeros_like(_to_gpu(b))
        rep = f.refine(_to_gpu(b), X, rtol=1e-13, maxit=40)
        assert rep.rel_residual <= 1e-13
        assert rep.history[0] < 1e-2, (mg, rep.history[0])
        assert np.linalg.norm(X.cpu().numpy().T - xd) / np.linalg.norm(xd) < 1e-11
        its[mg] = rep.iterations
    assert abs(its[0] - its[1]) <= 1


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_solve_apply_inverse_pair(R, name):
    """The mixed factor's solve sweeps in FP32 arithmetic on FP32 copies of its blocks, its apply in
    FP64: the two are inverses of each other to the FP32 solve's rounding (2^-24 times the sweeps'
    growth; 2.4e-7..2.7e-7 measured, held to 32 x 2^-24 = 1.9e-6), adjoints too, and the solve
    agrees with the FP64 refinement target to the factor's own accuracy."""
    pr = CASES[name]()
    tree = R.Tree(pr.points, pr.leaf)
    s = max(pr.s_cfg, tree.info(pr.k).s_req_mixed)
    f = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                 precision=R.RSRS_PREC_MIXED, seed=23)
    b = pr.rhs()
    for adj in (False, True):
        y = f.apply(f.solve(_to_gpu(b), adjoint=adj), adjoint=adj).cpu().numpy().T
        assert np.linalg.norm(y - b) / np.linalg.norm(b) < 32 * 2.0 ** -24, adj
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    x0 = f.solve(_to_gpu(b)).cpu().numpy().T
    assert np.linalg.norm(x0 - xd) / np.linalg.norm(xd) < 1e-2
