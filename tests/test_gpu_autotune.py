"""Launch shapes (rsrs_tune_t) and the autotuner.

Every tile shape of the tensor-core sampling product must give the sketches of the default shape
(the tiles change no element's sum) and FP32-level agreement with the FP64 product on ragged
sizes; the cluster-CPQR cluster and thread counts and the refinement residual's splits must give
factors and residuals that refine to the dense solution; the autotuner must return a valid
configuration, append it to its cache file and read it back without timing.
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


@pytest.mark.parametrize("d,kind,n,s", [(2, "log2d", 1000, 1100), (3, "invr3d", 777, 800), (2, "log2d", 21, 40),
                                        (2, "log2d", 200, 216)])
@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6, 7])
def test_sample_tiles_match_default_and_fp64(R, d, kind, n, s, tile):
    pts = W.uniform_points(n, d, W.rng_for(98, n, 1))
    rng = np.random.default_rng(n + 1)
    om = rng.standard_normal((n, s))
    ps = rng.standard_normal((n, s))
    t = R.Tree(pts, 4096)  # root is a leaf: the kept sketches are the sampled products
    out = {}
    for key, prec, tune in (("fp64", R.RSRS_PREC_FP64, None), ("default", R.RSRS_PREC_MIXED, None),
                            ("tile", R.RSRS_PREC_MIXED, {"sample_tile": tile})):
        f = R.Factor(t, R.kind_of(kind), 8, s, shift=1.0, scale=1.0 / n, precision=prec, omega=om, psi=ps,
                     keep_sketches=True, tune=tune)
        Y, Z, Om, Ps = f.sketches()
        out[key] = (Y - Om, Z - Ps)
    for a, b, c in zip(out["tile"], out["default"], out["fp64"]):
        scale = np.abs(c).max()
        assert np.abs(a - b).max() <= 1e-7 * scale
        assert np.abs(a - c).max() <= 1e-5 * scale


@pytest.mark.parametrize("tune", [{"cpqr_cluster": 4}, {"cpqr_cluster": 16, "cpqr_threads": 256},
                                  {"cpqr_threads": 512}, {"residual_split": 1}, {"residual_split": 16},
                                  {"sample_tile": 2, "cpqr_cluster": 8, "residual_split": 3}])
def test_tuned_factors_refine(R, tune):
    pr = W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=2, seed_problem=3)
    tree = R.Tree(pr.points, pr.leaf)
    s = tree.info(pr.k).s_req_mixed
    b = pr.rhs()
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    res = {}
    for key, tn in (("default", None), ("tuned", tune)):
        f = R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                     precision=R.RSRS_PREC_MIXED, seed=5, tune=tn)
        X = torch.zeros_like(_to_gpu(b))
        rep = f.refine(_to_gpu(b), X, rtol=1e-13, maxit=40)
        assert rep.rel_residual <= 1e-13
        assert rep.history[0] < 1e-2
        assert np.linalg.norm(X.cpu().numpy().T - xd) / np.linalg.norm(xd) < 1e-11
        Bg = _to_gpu(b)
        res[key] = f.residual(Bg, _to_gpu(xd), torch.empty_like(Bg)).cpu().numpy().T
    # the float-float residual of the dense solution, split or not, is at its rounding level
    nb = np.linalg.norm(b)
    assert np.linalg.norm(res["tuned"] - res["default"]) <= 1e-13 * nb


def test_autotune_cache_roundtrip(R, tmp_path):
    pr = W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=2, seed_problem=3)
    tree = R.Tree(pr.points, pr.leaf)
    s = tree.info(pr.k).s_req_mixed
    cache = str(tmp_path / "tune.txt")
    tune, rep = R.autotune(tree, R.RSRS_OP_LOG2D, pr.k, s, pr.diag_shift, pr.scale, reps=1, cache=cache)
    assert not rep["from_cache"] and rep["candidates"] >= 10
    assert 0 < rep["tuned_ms"] <= rep["default_ms"] * 1.05
    assert tune["sample_tile"] in (0, 1, 2, 3, 4, 5, 6, 7) and tune["cpqr_cluster"] in (0, 2, 4, 8, 16)
    again, rep2 = R.autotune(tree, R.RSRS_OP_LOG2D, pr.k, s, pr.diag_shift, pr.scale, reps=1, cache=cache)
    assert rep2["from_cache"] and rep2["candidates"] == 0 and again == tune
    with open(cache) as fh:
        assert len(fh.read().splitlines()) == 1
    f = R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                 precision=R.RSRS_PREC_MIXED, seed=5, tune=tune)
    b = pr.rhs()
    X = torch.zeros_like(_to_gpu(b))
    assert f.refine(_to_gpu(b), X, rtol=1e-13, maxit=40).rel_residual <= 1e-13


def test_autotune_batched(R):
    prs = [W.small_problem(n=n, d=2, leaf=24, k=10, nrhs=1, seed_problem=10 + i) for i, n in enumerate((1500, 2600))]
    trees = [R.Tree(p.points, p.leaf) for p in prs]
    s = max(t.info(10).s_req_mixed for t in trees)
    tune, rep = R.autotune(trees, [R.RSRS_OP_LOG2D] * 2, 10, s, [p.diag_shift for p in prs],
                           [p.scale for p in prs], reps=1)
    assert not rep["from_cache"] and rep["candidates"] > 0
    fs = R.build_batched(trees, [R.RSRS_OP_LOG2D] * 2, 10, s, [p.diag_shift for p in prs], [p.scale for p in prs],
                         precision=R.RSRS_PREC_MIXED, seed=9, tune=tune)
    for p, f in zip(prs, fs):
        b = p.rhs()
        X = torch.zeros_like(_to_gpu(b))
        assert f.refine(_to_gpu(b), X, rtol=1e-12, maxit=40).rel_residual <= 1e-12
