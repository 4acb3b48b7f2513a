"""Exact binary32 arithmetic for pinning the oracle.

Values are held as exact rationals (``fractions.Fraction``) and every operation
is rounded to the nearest binary32 value, ties to even, by integer arithmetic.
This is an independent route to the IEEE-754 result: it shares neither code
nor hardware rounding with the C oracle.
"""
from fractions import Fraction

import numpy as np

_MIN_EXP = -126          # smallest normal exponent
_MANT = 23               # fraction bits
_MAX = (2 - Fraction(1, 2 ** 23)) * Fraction(2) ** 127


def exact(v) -> Fraction:
    """Exact rational value of a binary32 (or Python float) number."""
    return Fraction(float(np.float32(v)))


def round_f32(v: Fraction) -> Fraction:
    """Round an exact rational to binary32, round-to-nearest, ties to even.
    Overflow returns +/-inf as a float."""
    if v == 0:
        return Fraction(0)
    sign = -1 if v < 0 else 1
    a = -v if v < 0 else v
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, _MIN_EXP)
    q = Fraction(2) ** (e - _MANT)
    m = a / q
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    r = fl * q
    if r > _MAX:
        return float("inf") if sign > 0 else float("-inf")
    return sign * r


def sqdist(qx, qy, px, py) -> Fraction:
    """d = dx*dx + dy*dy with dx = qx - px, dy = qy - py, each step rounded."""
    dx = round_f32(exact(qx) - exact(px))
    dy = round_f32(exact(qy) - exact(py))
    return round_f32(round_f32(dx * dx) + round_f32(dy * dy))


def sqdist_fused(qx, qy, px, py) -> Fraction:
    """The same expression evaluated as fma(dx, dx, dy*dy): one rounding fewer."""
    dx = round_f32(exact(qx) - exact(px))
    dy = round_f32(exact(qy) - exact(py))
    return round_f32(dx * dx + round_f32(dy * dy))


def to_f32(v: Fraction) -> np.float32:
    return np.float32(float(v))
