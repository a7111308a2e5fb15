"""The 7-point variable-coefficient operator (the PDE workload, given by its matvec only) through
the callback path: the device stencil against the oracle's, RSRS in FP64 against the oracle on the
same inputs, and the mixed factor refined with the callback's FP64 residual.

Sizes: a 12^3 grid with leaf 3^3 and k = 8 for parity (the oracle builds it in seconds), and the
32^3 grid with leaf 8^3 and k = 96 of the PDE workload reduced from 64^3 for the mixed path (s = the
mixed-precision sample bound, a little above s_req = 11,104), checked through the residual the
oracle's stencil computes exactly.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operators as ops
from oracle import rsrs as orsrs
from test_gpu_parity import AFTER_TIE, id_amplification, prior_amplifications, skeleton_parity, tie_band

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


def _stencil_problem(m, leaf, k, nrhs=2, problem=0):
    return W.Problem(name=f"stencil7_{m}cube", cfg=4, problem=problem, d=3, kernel="stencil7",
                     points=W.grid_points_3d(m), leaf=leaf, k=k, s_cfg=0, nrhs=nrhs, diag_shift=0.0,
                     scale=1.0, grid_side=m)


def _to_gpu(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a).T), device="cuda", dtype=torch.float64)


def _from_gpu(x):
    return x.cpu().numpy().T


@pytest.mark.parametrize("m", [5, 12])
def test_stencil_matvec_matches_oracle(R, m):
    pr = _stencil_problem(m, 27, 8)
    st = R.Stencil7(pr.coefficients(), m)
    x = np.random.default_rng(m).standard_normal((pr.n, 3))
    y = _from_gpu(st.matvec(_to_gpu(x), torch.empty((3, pr.n), device="cuda", dtype=torch.float64)))
    ref = ops.Stencil7Operator(m, pr.coefficients()).matvec(x)
    assert np.abs(y - ref).max() <= 1e-14 * np.abs(ref).max()


def test_stencil_rejects_bad_coefficients(R):
    with pytest.raises(R.RSRSError):
        R.Stencil7(np.full(27, -1.0), 3)


def test_stencil_fp64_matches_oracle(R):
    """The 12^3 operator in FP64 against the oracle on the same test matrices.  Skeletons must agree
    up to an accepted near-tie (tie_band: 1e-10 of |R_00|, or the nullification's rounding
    level for boxes whose far field is weak fill from eliminated neighbours).  Without a near-tie
    the unrefined solutions agree to 1e-10 or to the ID's measured amplification of the rounding
    (derived as in test_gpu_parity); after one, the two factorizations are different valid
    approximations, and the GPU's unrefined solution must be as accurate as the oracle's against
    the dense solution."""
    pr = _stencil_problem(12, 27, 8)
    trace = []
    tree_o, sched, fac, _ = orsrs.build(pr, trace=trace)
    st = R.Stencil7(pr.coefficients(), 12)
    t = R.Tree(pr.points, pr.leaf)
    f = R.Factor(t, R.RSRS_OP_CALLBACK, pr.k, fac.s, shift=0.0, scale=1.0, omega=pr.omega(fac.s),
                 psi=pr.psi(fac.s), matvec=st)
    assert f.stats().n_boxes == len(fac.boxes)
    tie = None
    prior = prior_amplifications(fac, trace)
    for i, bf in enumerate(fac.boxes):
        tie = skeleton_parity(f.box(i), bf, tie_band(bf, trace[i], fac.s, prior[i]))
        if tie is not None:
            print(f"stencil 12^3: tie at box {i} of {len(fac.boxes)} (amplification reaching it "
                  f"{prior[i]:.1e})")
            break
    b = pr.rhs()
    x = _from_gpu(f.solve(_to_gpu(b)))
    ref = orsrs.solve(fac, b)
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    if tie is None:
        tol = max(SOLVE_TOL, 1e-14 * id_amplification(fac, trace))
        e = np.linalg.norm(x - ref) / np.linalg.norm(ref)
        print(f"stencil 12^3: unrefined solutions agree to {e:.2e} (tolerance {tol:.1e})")
        assert e < tol
    else:
        e_gpu = np.linalg.norm(x - xd) / np.linalg.norm(xd)
        e_or = np.linalg.norm(ref - xd) / np.linalg.norm(xd)
        print(f"stencil 12^3 after a near-tie: unrefined errors gpu {e_gpu:.2e}, oracle {e_or:.2e}")
        assert e_gpu <= AFTER_TIE * e_or + 1e-13
    # the pair is an exact inverse on the device
    y = _from_gpu(f.apply(f.solve(_to_gpu(b))))
    assert np.linalg.norm(y - b) / np.linalg.norm(b) < 1e-12
    # refinement with the callback's residual reaches the dense solution
    X = torch.zeros_like(_to_gpu(b))
    rep = f.refine(_to_gpu(b), X, rtol=1e-13, maxit=40)
    assert rep.rel_residual <= 1e-13
    assert np.linalg.norm(_from_gpu(X) - xd) / np.linalg.norm(xd) < 1e-10


def test_stencil_mixed_refined_32cube(R):
    pr = _stencil_problem(32, 512, 96, nrhs=4)
    st = R.Stencil7(pr.coefficients(), 32)
    t = R.Tree(pr.points, pr.leaf)
    s = t.info(pr.k).s_req_mixed  # above s_req = 11,104: the FP32 near-field Grams need the margin
    f = R.Factor(t, R.RSRS_OP_CALLBACK, pr.k, s, shift=0.0, scale=1.0, precision=R.RSRS_PREC_MIXED, seed=3,
                 matvec=st)
    b = pr.rhs()
    X = torch.zeros_like(_to_gpu(b))
    rep = f.refine(_to_gpu(b), X, rtol=1e-12, maxit=60)
    assert rep.rel_residual <= 1e-12
    x = _from_gpu(X)
    r = b - ops.Stencil7Operator(32, pr.coefficients()).matvec(x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-11
