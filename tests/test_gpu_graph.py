"""Builds captured as one CUDA graph (opts.use_graph) and rebuilt in place by rsrs_refactor.

A graph build runs the same kernels in the same order as a plain build, so its factor must equal
the plain build's bit for bit (compared through solves); rsrs_refactor with a new seed must equal
a plain build with that seed, for FP64, mixed precision and batched builds.
"""
import numpy as np
import pytest

import workloads as W

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


@pytest.mark.parametrize("mixed", [False, True])
def test_graph_build_and_refactor_equal_plain_builds(R, mixed):
    pr = W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=3, seed_problem=3)
    tree = R.Tree(pr.points, pr.leaf)
    info = tree.info(pr.k)
    s = info.s_req_mixed if mixed else info.s_req
    prec = R.RSRS_PREC_MIXED if mixed else R.RSRS_PREC_FP64
    b = _to_gpu(pr.rhs())

    def plain(seed):
        f = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec,
                     seed=seed)
        return f.solve(b.clone())

    g = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=prec, seed=5,
                 use_graph=True)
    assert torch.equal(g.solve(b.clone()), plain(5))
    for seed in (9, 5, 123456789):
        g.refactor(seed)
        assert torch.equal(g.solve(b.clone()), plain(seed))
    X = torch.zeros_like(b)
    assert g.refine(b, X, rtol=1e-12, maxit=30).rel_residual <= 1e-12


def test_graph_batched_refactor(R):
    prs = [W.small_problem(n=1500, d=2, leaf=20, k=8, nrhs=2, seed_problem=11),
           W.small_problem(n=1100, d=3, kernel="invr3d", leaf=20, k=8, nrhs=2, seed_problem=12)]
    trees = [R.Tree(p.points, p.leaf) for p in prs]
    s = max(t.info(8).s_req for t in trees)
    kinds = [R.kind_of(p.kernel) for p in prs]
    args = (trees, kinds, 8, s, [p.diag_shift for p in prs], [p.scale for p in prs])
    g = R.build_batched(*args, seed=3, use_graph=True)
    g[1].refactor(40)  # rebuilds both problems of the batch
    ref = R.build_batched(*args, seed=40)
    for pr, fg, fr in zip(prs, g, ref):
        b = _to_gpu(pr.rhs())
        assert torch.equal(fg.solve(b.clone()), fr.solve(b.clone()))


def test_refactor_needs_a_graph_build(R):
    pr = W.small_problem(n_side=32, leaf=16, k=8, nrhs=1)
    tree = R.Tree(pr.points, pr.leaf)
    s = tree.info(pr.k).s_req
    f = R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale, seed=1)
    with pytest.raises(R.RSRSError) as e:
        f.refactor(2)
    assert e.value.name == "RSRS_E_INVAL"
    with pytest.raises(R.RSRSError):
        R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale, omega=pr.omega(s),
                 psi=pr.psi(s), use_graph=True)
