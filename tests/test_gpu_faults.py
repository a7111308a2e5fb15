"""Failure detection on the device without a GPU fault: every failure is made on purpose by an
input or a wait that cannot complete, comes back as a status code, and leaves the context usable.

* a bounded mbarrier wait that nothing completes (rsrs_wait_selftest with no arrival) expires and
  reports RSRS_E_TIMEOUT; the same wait with its arrival completes; likewise the grid-wide
  barrier of the fused solve sweeps with one of its two CTAs missing (rsrs_grid_wait_selftest);
* a matvec callback that returns an error aborts the build with RSRS_E_CALLBACK;
* a non-finite entry in the caller's test matrix reaches the pivot checks of the CPQR and LU
  kernels, which record it in the device status word (RSRS_E_NONFINITE or RSRS_E_SINGULAR); every
  kernel's control flow and indexing are independent of the values, so the build runs to its end;
* after each of these a normal build and solve on the same device still reach the dense solution.
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


def _problem():
    return W.small_problem(n_side=24, leaf=16, k=8)


def _assert_context_usable(R):
    """A fresh FP64 build and solve after the failure reach the dense solution."""
    pr = _problem()
    t = R.Tree(pr.points, pr.leaf)
    s = t.info(pr.k).s_req
    f = R.Factor(t, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale, seed=5)
    b = pr.rhs()
    X = torch.zeros((b.shape[1], pr.n), device="cuda", dtype=torch.float64)
    B = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
    rep = f.refine(B, X, rtol=1e-13, maxit=30)
    assert rep.rel_residual <= 1e-13
    xd = np.linalg.solve(ops.make_operator(pr).dense(), b)
    assert np.linalg.norm(X.cpu().numpy().T - xd) / np.linalg.norm(xd) < 1e-11


def test_bounded_wait_expires_with_status(R):
    with pytest.raises(R.RSRSError) as e:
        R.wait_selftest(1 << 12, arrive=False)
    assert e.value.name == "RSRS_E_TIMEOUT"
    R.wait_selftest(1 << 12, arrive=True)  # the same wait, completed by its arrival
    torch.cuda.synchronize()
    _assert_context_usable(R)


def test_grid_barrier_wait_expires_with_status(R):
    """The fused solve sweeps' grid-wide barrier: with one CTA missing, the other's bounded wait
    expires and reports RSRS_E_TIMEOUT; with both present it completes; the context stays usable
    (a refined solve through the fused sweeps afterwards reaches the dense solution)."""
    with pytest.raises(R.RSRSError) as e:
        R.grid_wait_selftest(1 << 12, arrive=False)
    assert e.value.name == "RSRS_E_TIMEOUT"
    R.grid_wait_selftest(1 << 12, arrive=True)
    torch.cuda.synchronize()
    _assert_context_usable(R)


def test_callback_error_aborts_build(R):
    pr = _problem()
    t = R.Tree(pr.points, pr.leaf)
    s = t.info(pr.k).s_req
    calls = []

    def failing(ctx, adjoint, n, ncols, x, ldx, y, ldy, stream):
        calls.append((adjoint, n, ncols))
        return 5

    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.RSRS_OP_CALLBACK, pr.k, s, shift=0.0, scale=1.0, matvec=failing, seed=1)
    assert e.value.name == "RSRS_E_CALLBACK"
    assert len(calls) == 1 and calls[0][1] == pr.n  # the build stopped at the first product
    _assert_context_usable(R)


def test_nonfinite_test_matrix_is_reported(R):
    pr = _problem()
    t = R.Tree(pr.points, pr.leaf)
    s = t.info(pr.k).s_req
    om, ps = pr.omega(s), pr.psi(s)
    om = np.array(om, copy=True)
    om[17, 3] = np.nan
    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.kind_of(pr.kernel), pr.k, s, shift=pr.diag_shift, scale=pr.scale, omega=om, psi=ps)
    assert e.value.name in ("RSRS_E_NONFINITE", "RSRS_E_SINGULAR")
    _assert_context_usable(R)
