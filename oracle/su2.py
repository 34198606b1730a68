"""SU(2) coupling coefficients for the oracle (Racah closed forms).

All angular momenta are passed doubled (tj = 2j, tm = 2m) so that they are integers.
Clebsch-Gordan <j1 m1 j2 m2 | J M> follows the Condon-Shortley convention used by
Eq. 22 of the paper; the 6-j symbol is the one of Eqs. 25-26.
"""
from functools import lru_cache
from fractions import Fraction
from math import factorial, sqrt


def _f(x2):
    # factorial of an integer given doubled; returns None for negative / odd
    if x2 < 0 or x2 % 2:
        return None
    return factorial(x2 // 2)


def _delta_sq(a, b, c):
    """Triangle coefficient squared (a+b-c)!(a-b+c)!(-a+b+c)!/(a+b+c+1)! as Fraction."""
    f1, f2, f3 = _f(a + b - c), _f(a - b + c), _f(-a + b + c)
    f4 = _f(a + b + c + 2)
    if None in (f1, f2, f3, f4):
        return None
    return Fraction(f1 * f2 * f3, f4)


def triangle(a, b, c):
    return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0


@lru_cache(maxsize=None)
def cg(tj1, tm1, tj2, tm2, tJ, tM):
    """<j1 m1 j2 m2 | J M> by Racah's single-sum formula."""
    if tm1 + tm2 != tM or not triangle(tj1, tj2, tJ):
        return 0.0
    if abs(tm1) > tj1 or abs(tm2) > tj2 or abs(tM) > tJ:
        return 0.0
    if (tj1 + tm1) % 2 or (tj2 + tm2) % 2 or (tJ + tM) % 2:
        return 0.0
    pre = Fraction(tJ + 1) * _delta_sq(tj1, tj2, tJ)
    pre *= Fraction(_f(tj1 + tm1) * _f(tj1 - tm1) * _f(tj2 + tm2) * _f(tj2 - tm2)
                    * _f(tJ + tM) * _f(tJ - tM))
    s = Fraction(0)
    for k in range(0, tj1 + tj2 + tJ + 2, 2):
        d = [k, tj1 + tj2 - tJ - k, tj1 - tm1 - k, tj2 + tm2 - k,
             tJ - tj2 + tm1 + k, tJ - tj1 - tm2 + k]
        if min(d) < 0:
            continue
        den = 1
        for x in d:
            den *= _f(x)
        s += Fraction((-1) ** (k // 2), den)
    val = float(s) * sqrt(float(pre))
    return val


@lru_cache(maxsize=None)
def sixj(a, b, c, d, e, f):
    """Wigner 6-j symbol {a b c; d e f} (all doubled) by Racah's formula."""
    for (x, y, z) in ((a, b, c), (a, e, f), (d, b, f), (d, e, c)):
        if not triangle(x, y, z):
            return 0.0
    pre = _delta_sq(a, b, c) * _delta_sq(a, e, f) * _delta_sq(d, b, f) * _delta_sq(d, e, c)
    s = Fraction(0)
    t_lo = max(a + b + c, a + e + f, d + b + f, d + e + c)
    t_hi = min(a + b + d + e, b + c + e + f, a + c + d + f)
    for t in range(t_lo, t_hi + 1, 2):
        num = _f(t + 2)
        den = (_f(t - a - b - c) * _f(t - a - e - f) * _f(t - d - b - f) * _f(t - d - e - c)
               * _f(a + b + d + e - t) * _f(b + c + e + f - t) * _f(a + c + d + f - t))
        s += Fraction((-1) ** (t // 2) * num, den)
    return float(s) * sqrt(float(pre))
