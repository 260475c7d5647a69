"""Pins of the oracle's stochastic rounding to bfloat16 (precision form: bf16
tables, float arithmetic, stochastic rounding on every store).

The oracle takes its 16 random bits as an input; these tests tie it to the
definition of stochastic rounding rather than to itself: over all 2^16 values
of the random bits exactly f * 2^16 round away from zero (f the fraction of
an ulp the value lies above its truncation), every result is one of the two
neighbours, bf16 values are fixed points, and over 10^6 keyed draws the mean
of the rounded values equals the input within 5 sigma.
"""
import struct

import numpy as np
import pytest


def f2b(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def b2f(b: int) -> float:
    return struct.unpack("<f", struct.pack("<I", b & 0xffffffff))[0]


def bf16_to_f64(h: np.ndarray) -> np.ndarray:
    return (h.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


# values spread over sign, magnitude, binade edges and subnormals
PATTERNS = [f2b(1 / 3), f2b(-2 / 3 * 2.0 ** -100), f2b(3.14159), 0x3f7fffff, 0xbf800001, 0x00012345,
            0x80000001, f2b(1.0 + 2.0 ** -20), f2b(-1234.5678), 0x7f7f8000]


@pytest.mark.parametrize("xb", PATTERNS)
def test_exhaustive_random_bits_give_the_fraction(orc, xb):
    """Over every 16-bit r, exactly (x & 0xffff) of them round away from zero,
    and every result is the truncation or the next pattern away from zero."""
    down = xb >> 16
    away = 0
    for r in range(1 << 16):
        h = orc.sr_bf16(xb, r)
        assert h in (down, (down + 1) & 0xffff), (hex(xb), r, hex(h))
        away += h != down
    assert away == (xb & 0xffff)


def test_neighbours_bracket_the_value(orc):
    """The two possible results bracket x on the real line (so a sign or
    direction error shows)."""
    for xb in PATTERNS[:-1]:
        x = b2f(xb)
        lo = b2f(orc.sr_bf16(xb, 0) << 16)
        hi = b2f(orc.sr_bf16(xb, 0xffff) << 16)
        assert min(lo, hi) <= x <= max(lo, hi)
        assert abs(lo) <= abs(x) <= abs(hi) or (xb & 0xffff) == 0


def test_bf16_values_are_fixed_points(orc):
    """Every finite bf16 pattern (and the infinities) rounds to itself under
    any key."""
    h = np.arange(1 << 16, dtype=np.uint32)
    finite = ((h >> 7) & 0xff) != 0xff
    inf = (h & 0x7fff) == 0x7f80
    keep = h[finite | inf]
    x = keep << 16
    for counter in range(8):
        out = orc.sr_bf16_row(x, 11, 3 + counter, counter)
        assert np.array_equal(out.astype(np.uint32), keep)


def test_nan_and_infinity(orc):
    assert orc.sr_bf16(0x7f800000, 0xffff) == 0x7f80
    assert orc.sr_bf16(0xff800000, 0xffff) == 0xff80
    for nan in (0x7fc00000, 0x7f800001, 0xff800001, 0x7fffffff):
        assert orc.sr_bf16(nan, 0x1234) == 0x7fc0


@pytest.mark.parametrize("xb", PATTERNS[:-1])
def test_unbiased_over_keyed_draws(orc, xb):
    """E[SR(x)] = x: the mean over 10^6 keyed draws (distinct element keys of
    the rounding stream) is within 5 sigma of x."""
    m = 1_000_000
    x = np.full(m, xb, np.uint32)
    out = orc.sr_bf16_row(x, 2024, 17, 5)
    vals = bf16_to_f64(out)
    xv = float(np.float32(b2f(xb)))
    lo = float(bf16_to_f64(np.array([xb >> 16], np.uint16))[0])
    hi = float(bf16_to_f64(np.array([(xb >> 16) + 1], np.uint16))[0])
    f = (xb & 0xffff) / 65536.0
    sigma = abs(hi - lo) * np.sqrt(f * (1 - f) / m)
    assert abs(vals.mean() - xv) <= 5 * sigma + 1e-300, (vals.mean(), xv, sigma)
    # rounding to nearest would be off by min(f, 1 - f) ulp: far outside 5 sigma
    # wherever the fraction is not within 1 % of a neighbour
    if 0.01 <= f <= 0.99:
        assert min(f, 1 - f) * abs(hi - lo) > 20 * sigma


def test_keyed_bits_are_the_rounding_stream(orc):
    """The keyed form takes word (element % 4) of Philox(seed; element / 4,
    row, counter, stream 4) -- the same counter layout as the other streams."""
    seed, row, counter = 99, 12, 3
    for element in range(8):
        w = orc.philox(seed, [element // 4, row, counter, orc.STREAM_SR])
        r16 = int(w[element % 4]) & 0xffff
        xb = 0x3eaaaaab
        assert orc.sr_bf16_keyed(xb, seed, element, row, counter) == orc.sr_bf16(xb, r16)


def test_sr_array_equals_scalar_definition(orc):
    """The array form applies the pinned scalar rounding element by element."""
    rng = np.random.default_rng(3)
    x = rng.integers(0, 1 << 32, size=4000, dtype=np.uint64).astype(np.uint32)
    r = rng.integers(0, 1 << 16, size=4000, dtype=np.uint64).astype(np.uint16)
    got = orc.sr_bf16_array(x, r)
    assert all(int(got[i]) == orc.sr_bf16(int(x[i]), int(r[i])) for i in range(x.size))
