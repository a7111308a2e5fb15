"""The FP64 <-> FP32 conversions the mixed path's sketch updates run on the integer pipes must equal
the hardware conversions bit for bit (IEEE 754 round to nearest, ties to even; exact widening),
on random values over the whole binary32 range and on the edge cases of the rounding: exact ties
(both parities), carries that reach the exponent, the largest finite binary32 and the overflow
threshold, the smallest normal and the subnormal range, signed zeros, infinities and NaN."""
import numpy as np
import pytest

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


def _inputs():
    rng = np.random.default_rng(2311)
    # random binary32 patterns (finite), widened, then perturbed inside and beyond one binary32 ulp
    bits = rng.integers(0, 2**31 - 1, size=200_000, dtype=np.int64).astype(np.uint32)
    bits = bits[(bits & 0x7F800000) != 0x7F800000]
    f = bits.view(np.float32).astype(np.float64) * np.where(rng.random(bits.size) < 0.5, -1.0, 1.0)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    cases = [
        f,
        f + ulp * rng.random(f.size),                      # between two binary32 values
        f + 0.5 * ulp,                                      # exact ties (even and odd last bit)
        f - 0.5 * ulp,
        f + 0.5 * ulp * (1 + 2.0**-29),                     # just above a tie
        rng.standard_normal(100_000) * 10.0 ** rng.integers(-40, 40, size=100_000),
    ]
    big = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edge = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0,
            np.nextafter(2.0, 0.0), 2.0 - 2.0**-25, 2.0 - 2.0**-24, 1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24,
            big, -big, big * (1 + 2.0**-25), big * (1 + 2.0**-24 - 2.0**-40), big * (1 + 2.0**-24), 1e39, -1e39,
            tiny, -tiny, tiny * (1 - 2.0**-25), tiny / 2, tiny * 2.0**-23, tiny * 2.0**-24, tiny * 2.0**-30,
            5e-324, -5e-324, 2.0**-1074 * 3, 1e-300]
    cases.append(np.array(edge))
    # mantissa all ones below each power of two: rounding carries into the exponent
    e = rng.integers(-125, 127, size=5_000).astype(np.float64)
    cases.append(2.0**e * (2.0 - 2.0**-30))
    # the binary32 subnormal range (results rounded to multiples of 2^-149, ties included)
    sub = rng.random(20_000) * tiny * np.where(rng.random(20_000) < 0.5, -1.0, 1.0)
    cases.append(sub)
    cases.append(np.array([2.0**-150, 3 * 2.0**-151, 2.0**-149, 1.5 * 2.0**-149, 2.5 * 2.0**-149,
                           tiny * (1 - 2.0**-25), tiny * (1 - 2.0**-24), tiny * (1 - 2.0**-23)]))
    return np.concatenate(cases)


def test_integer_pipe_conversions_match_the_hardware(R):
    x = torch.tensor(_inputs(), dtype=torch.float64, device="cuda")
    f, g = R.convert_selftest(x)
    torch.cuda.synchronize()
    ref_f = x.float()
    nan = torch.isnan(ref_f)
    assert torch.equal(torch.isnan(f), nan)
    diff = (f.view(torch.int32) != ref_f.view(torch.int32)) & ~nan
    assert int(diff.sum()) == 0, x[diff][:8].tolist()
    ref_g = f.double()
    nan_g = torch.isnan(ref_g)
    assert torch.equal(torch.isnan(g), nan_g)
    diff_g = (g.view(torch.int64) != ref_g.view(torch.int64)) & ~nan_g
    assert int(diff_g.sum()) == 0, f[diff_g][:8].tolist()
