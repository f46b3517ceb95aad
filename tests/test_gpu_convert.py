"""GPU: the integer binary32 <-> binary64 conversions the mixed-precision
kernels use in place of the hardware conversion instructions equal the
hardware conversions bit for bit - every binary32 pattern one way; every
binary32 value, every rounding midpoint between neighbouring binary32 values
and its two binary64 neighbours, and 2^28 pseudo-random binary64 patterns
the other way (IEEE 754 round to nearest, ties to even)."""
import pytest

pytestmark = pytest.mark.gpu


def test_integer_conversions_equal_hardware():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    r = G.selftest_conversions(n_random=1 << 28, seed=240408849)
    assert r["f2d"] == (1 << 32, 0)
    checked, bad = r["d2f"]
    # 4 checks per finite binary32 (value, midpoint and its two neighbours),
    # 1 per infinity / NaN pattern, plus the random patterns
    n_nonfinite = 2 * (1 << 23)
    assert checked == 4 * ((1 << 32) - n_nonfinite) + n_nonfinite + (1 << 28)
    assert bad == 0


def test_fma_reciprocal_within_one_ulp():
    """The column solve's reciprocal (approximate seed + one cubic
    Newton-Raphson step) stays within one ulp of the IEEE quotient 1.0 / x
    over 2^28 pseudo-random normal doubles of every sign and magnitude."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    checked, over, worst = G.selftest_reciprocal(n=1 << 28, seed=240408849)
    assert checked == 1 << 28
    assert over == 0 and worst <= 1


def test_double_float_split_bound():
    """The double-float split of GRIST_MIX_DF: h is x rounded to binary32
    (bit-exact against the hardware) and h + l is within 2^-47 |x|, over
    2^28 pseudo-random doubles of every sign and of magnitudes 2^-74..2^127."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    checked, bad = G.selftest_split(n=1 << 28, seed=240408849)
    assert checked == 1 << 28 and bad == 0
