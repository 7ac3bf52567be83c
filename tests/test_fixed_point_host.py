"""Host side of the exact gradient sums (no GPU): the 128-bit two's-complement
encoding that lt_gradient_fixed returns (low word, high word as int64), its
decoding into Python integers, and the conversion integer x 2^-64 / G to a
correctly rounded double, checked against exact rational arithmetic."""
from fractions import Fraction

import numpy as np

from paper_2310_02043_gb300.lighttrace import fixed_to_ints, gradient_from_fixed


def _encode(v: int):
    lo = v & ((1 << 64) - 1)
    return (lo - (1 << 64) if lo >= (1 << 63) else lo, v >> 64)


VALUES = [0, 1, -1, (1 << 64) - 1, -(1 << 64), (1 << 64) + 12345, -(1 << 100) - 7, (1 << 126) - 1, -(1 << 126),
          3 << 70, (1 << 117) + (1 << 64) + 1,        # sticky bit below the rounding position
          (1 << 117) + (1 << 64),                     # exact tie: rounds to even
          -((1 << 117) + (3 << 64))]                  # tie, odd: rounds away


def test_decoding_round_trips():
    sums = np.array([[_encode(v) for v in VALUES]], np.int64)
    ints = fixed_to_ints(sums)
    assert [int(x) for x in ints[0]] == VALUES


def test_conversion_is_correctly_rounded():
    sums = np.array([[_encode(v) for v in VALUES]], np.int64)
    for G in (1.0, 2.0 ** -37, 2.0 ** 20):
        g = gradient_from_fixed(sums, G)
        for v, x in zip(VALUES, g[0]):
            assert x == float(Fraction(v, 1 << 64) / Fraction(G)), (v, G)


def test_partition_sums_add_exactly():
    rng = np.random.default_rng(1)
    terms = [int(t) for t in rng.integers(-(1 << 62), 1 << 62, 1000)]
    whole = sum(terms)
    parts = [sum(terms[:300]), sum(terms[300:701]), sum(terms[701:])]
    enc = [np.array([[_encode(p)]], np.int64) for p in parts]
    total = sum(fixed_to_ints(e) for e in enc)
    assert int(total[0, 0]) == whole
    assert gradient_from_fixed(total, 0.5)[0, 0] == float(Fraction(whole, 1 << 64) * 2)
