"""The refinement residual R = B - A X (iterative refinement, an addition to the paper) in each of the
library's arithmetics against dense FP64: FP64, float-float on the FP32 pipe, and the Ozaki scheme on
the bf16 tensor cores (digits of K and X, exact integer sums).

B is taken as A X plus a perturbation of 1e-10, so R is about 1e-10 of B: the regime of iterative
refinement, where the residual is a small difference of large terms.  Every arithmetic must
reproduce the dense FP64 residual (numpy) to 2e-14 of |B| + |A||X| entry by entry.  A stress case
puts pairs of points 1e-7 and 1e-9 apart, so that a few rows' largest entries are far above their
typical ones (the Ozaki scheme scales each row by its largest entry); there float-float is held to
1e-13 (it reaches 4.4e-14 in 3D, the Ozaki scheme 1.6e-15).
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


def _close_pairs(n, d, kernel, seed):
    pts = W.uniform_points(n, d, W.rng_for(95, seed, 0))
    pts[1] = pts[0] + 1e-7 / np.sqrt(d)
    pts[3] = pts[2] + 1e-9 / np.sqrt(d)
    return W.kernel_problem(95, f"close_{kernel}", pts, kernel, 64, 16, 0, 4, problem=seed)


CASES = [
    ("grid2d_4096", lambda: W.config(0)[0], 1),
    ("rand2d_9000", lambda: W.small_problem(n=9000, d=2, leaf=64, k=16, nrhs=3, seed_problem=31), 3),
    ("rand2d_5000_20rhs", lambda: W.small_problem(n=5000, d=2, leaf=64, k=16, nrhs=20, seed_problem=32), 20),
    ("rand3d_4100", lambda: W.small_problem(n=4100, d=3, kernel="invr3d", leaf=64, k=16, nrhs=5,
                                            seed_problem=33), 5),
    ("close_pairs_2d_3000", lambda: _close_pairs(3000, 2, "log2d", 1), 4),
    ("close_pairs_3d_3000", lambda: _close_pairs(3000, 3, "invr3d", 2), 4),
]


def _to_gpu(a):
    return torch.tensor(np.ascontiguousarray(a.T), device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("name,make,nrhs", CASES, ids=[c[0] for c in CASES])
def test_residual_arithmetics_match_fp64(R, name, make, nrhs):
    pr = make()
    a = ops.make_operator(pr).dense()
    rng = np.random.default_rng(7)
    x = rng.standard_normal((pr.n, nrhs))
    b = a @ x + 1e-10 * rng.standard_normal((pr.n, nrhs))
    ref = b - a @ x
    scale = np.abs(b) + np.abs(a) @ np.abs(x)
    tree = R.Tree(pr.points, pr.leaf)
    s = tree.info(pr.k).s_req
    out = {}
    for mode in (R.RSRS_RESIDUAL_FP64, R.RSRS_RESIDUAL_FLOAT_FLOAT, R.RSRS_RESIDUAL_OZAKI):
        f = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale, seed=1,
                     residual=mode)
        Rr = torch.empty_like(_to_gpu(b))
        f.residual(_to_gpu(b), _to_gpu(x), Rr)
        out[mode] = Rr.cpu().numpy().T
    for mode, r in out.items():
        err = np.abs(r - ref) / scale
        print(f"{name}: residual arithmetic {mode}: largest error {err.max():.2e} of |b| + |A||x|")
        # float-float sums a row's terms in float-float with a fold every 256 terms; in 3D rows with a
        # neighbour at 1e-9 it keeps 4.4e-14 (measured), so it is held to 1e-13 in the stress cases
        bound = 1e-13 if (name.startswith("close") and mode == R.RSRS_RESIDUAL_FLOAT_FLOAT) else 2e-14
        assert err.max() < bound, (mode, err.max())
        # each resolves the 1e-10 perturbation (to about 1e-3 of itself); not in the stress cases,
        # where rows with entries of 1e9 / N make |A||x| (and so any arithmetic's rounding) larger
        if not name.startswith("close"):
            assert np.linalg.norm(r - ref) / np.linalg.norm(ref) < 1e-2


def test_refinement_uses_the_ozaki_residual_by_default(R):
    pr = W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=3, seed_problem=3)
    tree = R.Tree(pr.points, pr.leaf)
    s = tree.info(pr.k).s_req_mixed
    b = pr.rhs()
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    f = R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale, precision=R.RSRS_PREC_MIXED,
                 seed=5)
    X = torch.zeros_like(_to_gpu(b))
    rep = f.refine(_to_gpu(b), X, rtol=1e-13, maxit=40)
    assert rep.residual_kind == R.RSRS_RESIDUAL_OZAKI
    assert rep.rel_residual <= 1e-13
    assert np.linalg.norm(X.cpu().numpy().T - xd) / np.linalg.norm(xd) < 1e-11
    g = f.gmres(_to_gpu(b), torch.zeros_like(_to_gpu(b)), rtol=1e-12, restart=30, maxit=30)
    assert g.residual_kind == R.RSRS_RESIDUAL_OZAKI and g.rel_residual <= 1e-12
