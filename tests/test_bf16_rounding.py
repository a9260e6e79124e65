"""The FP32 -> BF16 rounding the 16-bit storage form uses (add 0x7FFF plus
the lowest kept bit, truncate 16 bits), checked against round-to-nearest,
ties-to-even to 8 significant bits computed independently in FP64."""
import numpy as np


def bias_truncate(x32):
    u = x32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFFFFFF
    return ((u >> 16) << 16).astype(np.uint32).view(np.float32)


def rne_reference(x32):
    x = x32.astype(np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    e = np.floor(np.log2(np.abs(x[nz])))
    q = np.exp2(e - 7)                  # spacing of 8-bit significands
    out[nz] = np.round(x[nz] / q) * q   # np.round: ties to even
    return out


def test_random_values_and_ties():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) *
         np.exp2(rng.integers(-40, 40, 200000))).astype(np.float32)
    # exact ties: kept 16 bits with a normal exponent (1..253, so that
    # rounding up stays finite), dropped bits exactly 0x8000; the random
    # 7-bit mantissa gives both parities of the kept lowest bit
    exp = rng.integers(1, 254, 10000).astype(np.uint32)
    mant = rng.integers(0, 128, 10000).astype(np.uint32)
    kept = (exp << 7) | mant
    ties = ((kept << 16) | 0x8000).view(np.float32)
    for v in (x, ties, -ties):
        got = bias_truncate(v).astype(np.float64)
        ref = rne_reference(v)
        # an exact-binade carry (e.g. 1.99.. -> 2.0) is still the RNE value
        np.testing.assert_array_equal(got, ref)


def test_overflow_rounds_to_infinity():
    big = np.array([np.finfo(np.float32).max], np.float32)
    assert np.isinf(bias_truncate(big))[0]
    assert bias_truncate(np.array([np.inf], np.float32))[0] == np.inf
