"""A float32 model of the digit split in the tensor-core operand writers (CPU).

The kernels that write bf16 digit planes split each symmetric residue s
(|s| ≤ (p − 1)/2 < 2^23) into signed digits in packed FP32:

* s itself: the float bits of 1.5·2^23 + s, minus 1.5·2^23, for p < 2^23;
  an exact int-to-float conversion above;
* byte digits: the carry q = floor((s + 128)/256) (a round-down FMA of
  (s + 128)·2^-8 onto 1.5·2^23, less 1.5·2^23), the digit s − 256·q;
* a balanced base b: q = fl(s·fl(1/b)) rounded to nearest (adding and taking
  off 1.5·2^23), the digit s − b·q.

These tests replay that arithmetic with numpy float32 (round to nearest, as
the kernels' rn instructions; the round-down step is taken by its
definition, floor, on exact values) and check that it reproduces the integer
split (the low byte read as signed, or the rounded float quotient) digit for
digit, within the bounds the library reports for the base it reports
(ffsyrk_digit_bounds, ffsyrk_digit_base), which size the accumulator units.
"""
import numpy as np
import pytest

from paper_2001_04109_gb300 import ffsyrk

MAGIC = np.float32(12582912.0)  # 1.5·2^23


def magic_to_float(s):
    """The float that the bits 0x4B400000 + s encode, less 1.5·2^23."""
    bits = (np.int64(0x4B400000) + s.astype(np.int64)).astype(np.uint32)
    return bits.view(np.float32) - MAGIC


def float_byte_split(s, D):
    """Byte digits as the kernels form them, from the exact float of s."""
    sf = s.astype(np.float32)
    assert np.array_equal(sf.astype(np.int64), s)  # |s| < 2^24: exact
    digits = []
    for _ in range(D - 1):
        u = sf + np.float32(128.0)
        scaled = u * np.float32(0.00390625)
        # both steps are exact: integers below 2^24, then a power-of-two scale
        assert np.array_equal(scaled.astype(np.float64), (sf.astype(np.float64) + 128.0) / 256.0)
        q = np.floor(scaled.astype(np.float64)).astype(np.float32)  # the round-down FMA onto 1.5·2^23
        d = sf - np.float32(256.0) * q  # exact: integers below 2^24
        digits.append(d.astype(np.int64))
        sf = q
    digits.append(sf.astype(np.int64))
    return digits


def int_byte_split(s, D):
    """The integer split: the low byte read as signed, the rest carried on."""
    digits = []
    for _ in range(D - 1):
        d = ((s & 0xFF) ^ 0x80) - 0x80
        digits.append(d)
        s = (s - d) >> 8
    digits.append(s)
    return digits


def test_magic_conversion_is_exact_below_2_22_only():
    s = np.arange(-(1 << 22) + 1, 1 << 22, 997, dtype=np.int64)
    s = np.concatenate([s, [-(1 << 22) + 1, -1, 0, 1, (1 << 22) - 1]])
    assert np.array_equal(magic_to_float(s).astype(np.int64), s)
    # past 2^22 the sum leaves 1.5·2^23's binade: the writers convert s exactly instead
    big = np.array([(1 << 22) + 1, (1 << 23) - 1, -(1 << 22) - 1], dtype=np.int64)
    assert not np.array_equal(magic_to_float(big).astype(np.int64), big)


@pytest.mark.parametrize("p", [8388593, 16777213, 131357, 65521])
def test_byte_digits_match_the_integer_split(p):
    assert ffsyrk.digit_base(p) == 256
    bounds = ffsyrk.digit_bounds(p)
    D = len(bounds)
    H = (p - 1) // 2
    if H < 1 << 21:
        s = np.arange(-H, H + 1, dtype=np.int64)
    else:  # every residue near both ends and around each carry, a sample between
        rng = np.random.default_rng(p)
        ends = np.concatenate([np.arange(-H, -H + 70000), np.arange(H - 70000, H + 1)])
        ties = np.arange(-H // 256, H // 256 + 1, 37)[:, None] * 256 + np.array([127, 128, 129, -128, -129])
        s = np.concatenate([ends, ties.ravel(), rng.integers(-H, H + 1, 2_000_000)])
        s = s[np.abs(s) <= H].astype(np.int64)
    got = float_byte_split(s, D)
    want = int_byte_split(s.copy(), D)
    for t in range(D):
        assert np.array_equal(got[t], want[t]), f"digit {t}"
        assert np.abs(got[t]).max() <= bounds[t], f"digit {t} beyond its bound {bounds[t]}"
    recon = sum(got[t] * 256 ** t for t in range(D))
    assert np.array_equal(recon, s)


@pytest.mark.parametrize("p", [70001, 100003, 131063, 131071, 131101])
def test_balanced_digits_match_the_rounded_quotient(p):
    b = ffsyrk.digit_base(p)
    assert b != 256
    bounds = ffsyrk.digit_bounds(p)
    assert len(bounds) == 2
    H = (p - 1) // 2
    s = np.arange(-H, H + 1, dtype=np.int64)
    sf = s.astype(np.float32)
    dinv = np.float32(1.0) / np.float32(b)
    x = sf * dinv  # fl(s·fl(1/b))
    q = (x + MAGIC) - MAGIC  # rounded to nearest, ties to even, as the writers do it
    assert np.array_equal(q, np.rint(x))  # the integer path's float-to-int rounding
    d = sf - np.float32(b) * q
    assert np.array_equal(d.astype(np.int64), s - b * q.astype(np.int64))  # exact
    assert np.abs(d).max() <= bounds[0]
    assert np.abs(q).max() <= bounds[1]
