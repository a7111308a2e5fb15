"""Batched builds (independent problems in one set of launches) and the device test-matrix draws.

The device draws Omega / Psi with Philox4x32-10 and Box-Muller; ``workloads.philox_gaussian`` is the
same published generator in numpy (pinned to the Random123 known-answer vectors on the CPU), so the
oracle can be run on exactly the draws the device made.  Problem p of a batch uses key seed + p.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as ops
from oracle import rsrs as orsrs
from test_gpu_parity import AFTER_TIE, prior_amplifications, skeleton_parity, tie_band

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-10


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


def _from_gpu(x):
    return x.cpu().numpy().T


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _skeletons_agree(gpu_box, bf, band):
    """Identical skeleton lists, or a first difference that is an accepted near-tie (False)."""
    return skeleton_parity(gpu_box, bf, band) is None


def _problems():
    return [
        W.small_problem(n=1500, d=2, leaf=20, k=8, nrhs=2, seed_problem=11),
        W.small_problem(n_side=32, leaf=16, k=8, nrhs=2),
        W.small_problem(n=1100, d=3, kernel="invr3d", leaf=20, k=8, nrhs=2, seed_problem=12),
        W.small_problem(n=40, d=2, leaf=64, k=8, nrhs=2, seed_problem=13),  # root-only tree
    ]


SEED = 1234


@pytest.fixture(scope="module")
def batch(R):
    prs = _problems()
    trees = [R.Tree(p.points, p.leaf) for p in prs]
    k = prs[0].k
    s = max(t.info(k).s_req for t in trees)
    kinds = [R.kind_of(p.kernel) for p in prs]
    fs = R.build_batched(trees, kinds, k, s, [p.diag_shift for p in prs], [p.scale for p in prs],
                         precision=R.RSRS_PREC_FP64, seed=SEED)
    return prs, trees, k, s, kinds, fs


def test_device_draws_follow_the_counter_generator(R, batch):
    """Each batched factor against the oracle run on the device's own draws (key seed + p)."""
    prs, trees, k, s, kinds, fs = batch
    for p, (pr, f) in enumerate(zip(prs, fs)):
        om = W.philox_gaussian(pr.n, s, SEED + p, 0)
        ps = W.philox_gaussian(pr.n, s, SEED + p, 1)
        trace = []
        _, _, fac, _ = orsrs.build(pr, omega=om, psi=ps, s=s, trace=trace)
        assert f.stats().n_boxes == len(fac.boxes)
        prior = prior_amplifications(fac, trace)
        same = True
        for i, bf in enumerate(fac.boxes):
            if not _skeletons_agree(f.box(i), bf, tie_band(bf, trace[i], s, prior[i])):
                same = False
                break
        b = pr.rhs()
        xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
        for adj in (False, True):
            x = _from_gpu(f.solve(_to_gpu(b), adjoint=adj))
            ref = orsrs.solve(fac, b, adjoint=adj)
            if same:
                assert _rel(x, ref) < SOLVE_TOL, f"problem {p} adjoint={adj}"
            elif not adj:  # after a near-tie: as accurate as the oracle's factor (test_gpu_parity)
                assert _rel(x, xd) <= AFTER_TIE * _rel(ref, xd) + 1e-13, f"problem {p}"


def test_batched_matches_single_builds(R, batch):
    prs, trees, k, s, kinds, fs = batch
    for p, (pr, t, f) in enumerate(zip(prs, trees, fs)):
        g = R.Factor(t, kinds[p], k, s, shift=pr.diag_shift, scale=pr.scale, precision=R.RSRS_PREC_FP64,
                     seed=SEED + p)
        sb, sg = f.stats(), g.stats()
        assert sb.n_boxes == sg.n_boxes and sb.root_size == sg.root_size
        for i in range(sg.n_boxes):
            assert np.array_equal(f.box(i)["S"], g.box(i)["S"])
        assert np.array_equal(f.root()[0], g.root()[0])
        b = _to_gpu(pr.rhs())
        assert float(torch.linalg.norm(f.solve(b.clone()) - g.solve(b.clone())) / torch.linalg.norm(b)) < 1e-13
        assert float(torch.linalg.norm(f.apply(b.clone()) - g.apply(b.clone())) / torch.linalg.norm(b)) < 1e-13


def test_batched_matvec_and_refine(R, batch):
    prs, trees, k, s, kinds, fs = batch
    for pr, f in zip(prs, fs):
        b = pr.rhs()
        a = ops.make_operator(pr).dense()
        y = _from_gpu(f.matvec(_to_gpu(b), torch.empty_like(_to_gpu(b))))
        assert _rel(y, a @ b) < 1e-13
        X = torch.zeros_like(_to_gpu(b))
        rep = f.refine(_to_gpu(b), X, rtol=1e-13, maxit=30)
        assert rep.rel_residual <= 1e-13
        assert _rel(_from_gpu(X), np.linalg.solve(a, b)) < 1e-11


def test_batched_mixed_precision_refines(R):
    prs = _problems()
    trees = [R.Tree(p.points, p.leaf) for p in prs]
    k = prs[0].k
    s = max(t.info(k).s_req for t in trees)
    for sk in (1, 2):
        fs = R.build_batched(trees, [R.kind_of(p.kernel) for p in prs], k, s, [p.diag_shift for p in prs],
                             [p.scale for p in prs], precision=R.RSRS_PREC_MIXED, seed=77, sample_kernel=sk)
        for pr, f in zip(prs, fs):
            b = pr.rhs()
            X = torch.zeros_like(_to_gpu(b))
            rep = f.refine(_to_gpu(b), X, rtol=1e-12, maxit=30)
            assert rep.rel_residual <= 1e-12
            assert rep.history[0] < 1e-2  # the unrefined mixed factor: about 1e-3 (FP32 cancellation in the nullification)
            assert _rel(_from_gpu(X), np.linalg.solve(ops.make_operator(pr).dense(), b)) < 1e-10


def test_batched_rejects_mismatched_arguments(R):
    prs = _problems()[:2]
    trees = [R.Tree(p.points, p.leaf) for p in prs]
    s = max(t.info(8).s_req for t in trees)
    with pytest.raises(R.RSRSError):
        R.build_batched(trees, [R.RSRS_OP_LOG2D] * 2, 8, s - 1, [1.0, 1.0], [1e-3, 1e-3])
    with pytest.raises(R.RSRSError):
        R.build_batched(trees, [R.RSRS_OP_LOG2D] * 2, 0, s, [1.0, 1.0], [1e-3, 1e-3])
