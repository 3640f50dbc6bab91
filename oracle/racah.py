"""Exact Wigner-3j symbols from the Racah sum, in rational arithmetic.

TEST INFRASTRUCTURE ONLY (a second oracle for small multipoles).  Every
squared 3j symbol is rational, so this module returns the square as a
``fractions.Fraction`` together with the sign; nothing is rounded.  It backs
the Schulten-Gordon oracle in ``coupling_oracle.c`` for l <= 40 and supplies
the exact (0 0 0) closed form of the paper (Eqs. 000_sq_main and gdef, after
Edmonds 1957 Eq. 3.7.17) at any l.
"""
from fractions import Fraction
from math import comb, factorial


def _delta(j1, j2, j3):
    return Fraction(factorial(j1 + j2 - j3) * factorial(j1 - j2 + j3) * factorial(-j1 + j2 + j3),
                    factorial(j1 + j2 + j3 + 1))


def threej_exact(j1, j2, j3, m1, m2, m3):
    """(j1 j2 j3; m1 m2 m3) as (sign, square) with square a Fraction.

    Racah's single-sum formula: the symbol is
    (-1)^(j1-j2-m3) sqrt(Delta) sqrt(prod of (j+-m)!) * sum_k (-1)^k / D_k,
    D_k = k! (j3-j2+k+m1)! (j3-j1+k-m2)! (j1+j2-j3-k)! (j1-k-m1)! (j2-k+m2)!.
    Integer arguments only.  Returns (0, Fraction(0)) outside the selection
    rules.
    """
    if m1 + m2 + m3 != 0:
        return 0, Fraction(0)
    if any(abs(m) > j for j, m in ((j1, m1), (j2, m2), (j3, m3))):
        return 0, Fraction(0)
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0, Fraction(0)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    total = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (factorial(k) * factorial(j3 - j2 + k + m1) * factorial(j3 - j1 + k - m2) *
               factorial(j1 + j2 - j3 - k) * factorial(j1 - k - m1) * factorial(j2 - k + m2))
        total += Fraction((-1) ** k, den)
    if total == 0:
        return 0, Fraction(0)
    pref = (factorial(j1 + m1) * factorial(j1 - m1) * factorial(j2 + m2) * factorial(j2 - m2) *
            factorial(j3 + m3) * factorial(j3 - m3))
    square = _delta(j1, j2, j3) * pref * total * total
    sign = (-1) ** ((j1 - j2 - m3) % 2) * (1 if total > 0 else -1)
    return sign, square


def threej_float(j1, j2, j3, m1, m2, m3):
    """The exact symbol rounded once to a Python float (square root of the
    exact square, correctly rounded to double before the root)."""
    sign, sq = threej_exact(j1, j2, j3, m1, m2, m3)
    if sign == 0:
        return 0.0
    return sign * float(sq) ** 0.5


def g_exact(p):
    """g(p) = (2p)! / (2^(2p) (p!)^2) = C(2p, p) / 4^p (Eq. gdef), exact."""
    if p < 0:
        return Fraction(0)
    return Fraction(comb(2 * p, p), 4 ** p)


def threej000_sq_closed(j1, j2, j3):
    """(j1 j2 j3; 0 0 0)^2 = g(p1) g(p2) g(p3) / ((J+1) g(p)) for even J,
    0 for odd J (Eq. 000_sq_main with the halved triangle variables of
    Eq. trianglecombos).  Exact."""
    J = j1 + j2 + j3
    if J % 2 or j3 < abs(j1 - j2) or j3 > j1 + j2:
        return Fraction(0)
    p = J // 2
    p1, p2, p3 = (-j1 + j2 + j3) // 2, (j1 - j2 + j3) // 2, (j1 + j2 - j3) // 2
    return g_exact(p1) * g_exact(p2) * g_exact(p3) / ((J + 1) * g_exact(p))
