"""The refinement residual R = B - A X (iterative refinement, an addition to the paper) in float-float
arithmetic against FP64.

B is taken as A X plus a perturbation of 1e-10, so R is about 1e-10 of B: the regime of iterative
refinement, where the residual is a small difference of large terms.  The float-float product
must reproduce the dense FP64 residual (numpy) to about 1e-14 of |B| + |A||X| entry by entry, as
the FP64 kernel does.
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


CASES = [
    ("grid2d_4096", lambda: W.config(0)[0], 1),
    ("rand2d_9000", lambda: W.small_problem(n=9000, d=2, leaf=64, k=16, nrhs=3, seed_problem=31), 3),
    ("rand2d_5000_20rhs", lambda: W.small_problem(n=5000, d=2, leaf=64, k=16, nrhs=20, seed_problem=32), 20),
    ("rand3d_4100", lambda: W.small_problem(n=4100, d=3, kernel="invr3d", leaf=64, k=16, nrhs=5,
                                            seed_problem=33), 5),
]


def _to_gpu(a):
    return torch.tensor(np.ascontiguousarray(a.T), device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("name,make,nrhs", CASES, ids=[c[0] for c in CASES])
def test_float_float_residual_matches_fp64(R, name, make, nrhs):
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
    for fp64 in (False, True):
        f = R.Factor(tree, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale, seed=1,
                     residual_fp64=fp64)
        Rr = torch.empty_like(_to_gpu(b))
        f.residual(_to_gpu(b), _to_gpu(x), Rr)
        out[fp64] = Rr.cpu().numpy().T
    for fp64, r in out.items():
        err = np.abs(r - ref) / scale
        assert err.max() < 2e-14, (fp64, err.max())
    # the float-float residual resolves the 1e-10 perturbation (to about 1e-3 of itself)
    assert np.linalg.norm(out[False] - ref) / np.linalg.norm(ref) < 1e-2
