"""rsrs_solve_noalloc against rsrs_solve.

The no-allocation solve stages the right-hand sides in the library's static device buffer instead
of a per-call allocation (rsrs_solve's stream-ordered scratch); it runs the same kernels in the same order, so its results must equal
rsrs_solve's bit for bit, also for two calls in a row that reuse the buffer, and it must keep
working when no device memory can be allocated at all.  This file is named to be collected last,
so that it also runs after everything else has used the device.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ELEMS = 1 << 20  # RSRS_NOALLOC_MAX_ELEMS


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2311_01451_gb300 as pkg

    return pkg


@pytest.fixture(scope="module", params=["fp64", "mixed"])
def factor(R, request):
    """An FP64 factor (FP64 sweeps) and a mixed-precision one (FP32 sweeps through the second static
    buffer)."""
    pr = W.small_problem(n=3000, d=2, leaf=24, k=10, nrhs=3, seed_problem=3)
    tree = R.Tree(pr.points, pr.leaf)
    mixed = request.param == "mixed"
    s = tree.info(pr.k).s_req_mixed if mixed else tree.info(pr.k).s_req
    f = R.Factor(tree, R.RSRS_OP_LOG2D, pr.k, s, shift=pr.diag_shift, scale=pr.scale,
                 precision=R.RSRS_PREC_MIXED if mixed else R.RSRS_PREC_FP64, seed=5)
    return pr, f


def _block(n, nrhs, seed):
    g = np.random.default_rng(seed).standard_normal((nrhs, n))
    return torch.tensor(g, device="cuda", dtype=torch.float64)  # (nrhs, N): column-major N x nrhs


def test_noalloc_equals_solve_two_calls_in_a_row(R, factor):
    pr, f = factor
    F1, F2 = _block(pr.n, 3, 1), _block(pr.n, 5, 2)
    ref1 = f.solve(F1.clone())
    ref2 = f.solve(F2.clone(), adjoint=True)
    G1, G2 = F1.clone(), F2.clone()
    f.solve_noalloc(G1)
    f.solve_noalloc(G2, adjoint=True)  # reuses the staging buffer right after the first call
    torch.cuda.synchronize()
    assert torch.equal(G1, ref1)
    assert torch.equal(G2, ref2)
    # and again, in the opposite order
    H2, H1 = F2.clone(), F1.clone()
    f.solve_noalloc(H2, adjoint=True)
    f.solve_noalloc(H1)
    torch.cuda.synchronize()
    assert torch.equal(H1, ref1) and torch.equal(H2, ref2)


def test_noalloc_rejects_blocks_beyond_the_buffer(R, factor):
    pr, f = factor
    nrhs = MAX_ELEMS // pr.n + 1
    F = _block(pr.n, nrhs, 3)
    before = F.clone()
    with pytest.raises(R.RSRSError) as e:
        f.solve_noalloc(F)
    assert e.value.name == "RSRS_E_INVAL" and "exceeds" in str(e.value)
    torch.cuda.synchronize()
    assert torch.equal(F, before)  # nothing was launched


def test_noalloc_solves_with_device_memory_exhausted(R, factor):
    """The reason the entry point exists: a caller whose device memory is all held by another
    allocator.  Here PyTorch's allocator takes every block it can get; rsrs_solve then cannot obtain
    its staging block and reports RSRS_E_NOMEM (a host-side error, nothing is launched), while
    rsrs_solve_noalloc still solves, bit-identical to a solve made before the memory was taken."""
    pr, f = factor
    nrhs = 200  # 3000 x 200 doubles = 4.8 MB: within the static buffer, beyond what is left below
    F = _block(pr.n, nrhs, 4)
    ref = f.solve(F.clone())
    warm = F.clone()
    f.solve_noalloc(warm)  # the first call on the device resolves the buffer's address
    G, H = F.clone(), F.clone()
    torch.cuda.synchronize()
    hold = []
    try:
        # PyTorch serves requests above 1 MiB from segments of at least 2 MiB (20 MiB between 1 and
        # 10 MiB) and smaller ones from 2 MiB segments: the last, sub-MiB chunks leave < 2 MiB
        for chunk in (1 << 30, 1 << 26, 1 << 24, 1 << 19):
            while True:
                try:
                    hold.append(torch.empty(chunk, dtype=torch.uint8, device="cuda"))
                except torch.cuda.OutOfMemoryError:
                    break
        free, _ = torch.cuda.mem_get_info()
        assert free < F.numel() * 8, f"{free} bytes still free"
        with pytest.raises(R.RSRSError) as e:
            f.solve(H)
        assert e.value.name == "RSRS_E_NOMEM"
        f.solve_noalloc(G)
        torch.cuda.synchronize()
    finally:
        del hold
        torch.cuda.empty_cache()
    assert torch.equal(G, ref)  # compared once the memory is back (the comparison allocates)
