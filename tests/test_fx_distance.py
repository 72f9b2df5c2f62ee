"""Exactness of the covariance assembly's fixed-point squared distances (host run of the kernels'
integer routines through gp_debug_fx_sqdist).

The routine forms sum_d (qa_d - qb_d)^2 in 128-bit integers and rounds s 2^-twoF once to FP64 (nearest,
ties to even). The reference is Python's exact integer arithmetic and its correctly rounded conversion
of the exact rational s / 2^twoF to float: the two must agree bit for bit — on random coordinates of
every magnitude up to the 2^58 limit, on D up to 256, on scales across the whole exponent range, and on
constructed ties in both rounding directions.
"""
import ctypes
import math
from fractions import Fraction

import numpy as np
import pytest

import __graft_entry__
from paper_2602_19683_gb300 import _native as N

LIM = 1 << 58


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return N.load()


def fx(lib, qa, qb, twoF):
    a = (ctypes.c_int64 * len(qa))(*qa)
    b = (ctypes.c_int64 * len(qb))(*qb)
    out = ctypes.c_double()
    st = lib.gp_debug_fx_sqdist(a, b, len(qa), twoF, ctypes.byref(out))
    return st, out.value


def exact(qa, qb, twoF):
    s = sum((x - y) * (x - y) for x, y in zip(qa, qb))
    return float(Fraction(s, 1) / Fraction(2) ** twoF) if twoF >= 0 else float(s * 2 ** (-twoF))


@pytest.mark.parametrize("D", [1, 3, 8, 16, 256])
def test_random_coordinates_round_exactly(lib, D):
    rng = np.random.default_rng(D)
    for k in range(300):
        bits = int(rng.integers(1, 59))
        qa = [int(v) for v in rng.integers(-(1 << bits) + 1, 1 << bits, D, dtype=np.int64)]
        qb = [int(v) for v in rng.integers(-(1 << bits) + 1, 1 << bits, D, dtype=np.int64)]
        twoF = int(rng.integers(-800, 1023))
        st, got = fx(lib, qa, qb, twoF)
        assert st == N.GP_OK
        want = exact(qa, qb, twoF)
        assert got == want, (D, k, bits, twoF, got, want)


def test_ties_round_to_even(lib):
    # s = 2^60 + 128: the 53-bit mantissa ends at bit 8, the rest is exactly half an ulp, even -> down
    st, got = fx(lib, [1 << 30, 8, 8], [0, 0, 0], 0)
    assert st == N.GP_OK and got == float(1 << 60)
    # s = 2^60 + 256 + 128: same tie with the mantissa's last bit set -> up to 2^60 + 512
    st, got = fx(lib, [1 << 30, 16, 8, 8], [0, 0, 0, 0], 0)
    assert st == N.GP_OK and got == float((1 << 60) + 512)
    # just above half: s = 2^60 + 129 -> up
    st, got = fx(lib, [1 << 30, 8, 8, 1], [0, 0, 0, 0], 0)
    assert st == N.GP_OK and got == float((1 << 60) + 256)


def squares_summing_to(s, terms=16):
    """Integers whose squares sum to s (greedy, largest square first)."""
    out = []
    while s > 0 and len(out) < terms:
        r = math.isqrt(s)
        out.append(r)
        s -= r * r
    assert s == 0
    return out


def test_mantissa_carry_on_rounding_up(lib):
    # s = 2^54 - 1: 54 ones, the dropped bit is exactly half and the kept mantissa odd -> rounds up
    # to 2^54, carrying out of the 53-bit mantissa into the exponent
    t = squares_summing_to((1 << 54) - 1)
    st, got = fx(lib, t, [0] * len(t), 0)
    assert st == N.GP_OK and got == float(1 << 54)
    st, got = fx(lib, t, [0] * len(t), 10)
    assert st == N.GP_OK and got == float(1 << 44)


def test_extremes_and_rejections(lib):
    big = LIM - 1
    st, got = fx(lib, [big] * 256, [-big] * 256, 1022)
    assert st == N.GP_OK and got == exact([big] * 256, [-big] * 256, 1022)
    st, got = fx(lib, [5, -7], [5, -7], 100)
    assert st == N.GP_OK and got == 0.0
    assert fx(lib, [LIM], [0], 0)[0] == N.GP_ERR_INVALID_ARG
    assert fx(lib, [0], [0], 1023)[0] == N.GP_ERR_INVALID_ARG
    assert lib.gp_debug_fx_sqdist(None, None, 1, 0, None) == N.GP_ERR_INVALID_ARG
