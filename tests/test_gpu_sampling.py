"""Sampling kernels of the mixed path against the FP64 product (eq. rand_sample_setting).

A tree whose root is a leaf compresses nothing, so the kept sketches are exactly the sampled
Y = A Omega and Z = A* Psi.  The FP32 SIMT and the 3xTF32 tensor-core kernels must agree with
the FP64 kernel on the kernel part A - I to FP32-level accuracy (1e-5 relative), on ragged
sizes (rows not a multiple of 128, points not a multiple of 32 or of 4, a single partial chunk of
points, and 2s columns [Omega Psi] ending in a partial tile of every width class).
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


@pytest.mark.parametrize("d,kind,n,s", [(2, "log2d", 1000, 1100), (3, "invr3d", 777, 800), (2, "log2d", 257, 300),
                                        (2, "log2d", 21, 40), (3, "invr3d", 120, 132)])
@pytest.mark.parametrize("kernel", [1, 2])
def test_mixed_sampling_matches_fp64(R, d, kind, n, s, kernel):
    pts = W.uniform_points(n, d, W.rng_for(98, n, 0))
    rng = np.random.default_rng(n)
    om = rng.standard_normal((n, s))
    ps = rng.standard_normal((n, s))
    t = R.Tree(pts, 4096)
    assert t.info(8).depth == 0
    out = {}
    for prec, sk in ((R.RSRS_PREC_FP64, 0), (R.RSRS_PREC_MIXED, kernel)):
        f = R.Factor(t, R.kind_of(kind), 8, s, shift=1.0, scale=1.0 / n, precision=prec, omega=om, psi=ps,
                     keep_sketches=True, sample_kernel=sk)
        Y, Z, Om, Ps = f.sketches()
        out[prec] = (Y - Om, Z - Ps)
        assert np.array_equal(Om, om)
    for a, b in zip(out[R.RSRS_PREC_MIXED], out[R.RSRS_PREC_FP64]):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < 1e-5, err


@pytest.mark.parametrize("n,s", [(300, 320), (257, 301)])
def test_device_draws_match_counter_generator(R, n, s):
    """Omega and Psi drawn on the device (Philox4x32-10 + Box-Muller; one thread per pair when s is
    even, per entry when odd) equal workloads.philox_gaussian entry by entry, up to the last-bit
    differences of the FP64 log / sine / cosine of the two math libraries."""
    pts = W.uniform_points(n, 2, W.rng_for(97, n, 3))
    t = R.Tree(pts, 4096)
    f = R.Factor(t, R.RSRS_OP_LOG2D, 8, s, shift=1.0, scale=1.0 / n, seed=77, keep_sketches=True)
    _, _, Om, Ps = f.sketches()
    for got, stream in ((Om, 0), (Ps, 1)):
        ref = W.philox_gaussian(n, s, 77, stream)
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
