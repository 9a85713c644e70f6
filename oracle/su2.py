"""SU(2) coupling coefficients, exact rational arithmetic, FP64 results.

Oracle module (test infrastructure only).  All spins are passed as *twos*
(the integer 2j).  Pins: ``tests/test_oracle_su2.py`` checks the 6j against
closed forms, orthogonality and the 24 tetrahedral symmetries, and against a
6j computed from Clebsch-Gordan sums; the 9j against its zero-entry reduction,
orthogonality and a Clebsch-Gordan brute force; C~ against C~=1 for scalar
operators and against the m-resolved expansion in ``expand``.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache


def fact(n2: int) -> int:
    """(n2/2)! for an even twos argument."""
    assert n2 % 2 == 0 and n2 >= 0, n2
    return math.factorial(n2 // 2)


def triangle(a: int, b: int, c: int) -> bool:
    """|a-b| <= c <= a+b and a+b+c integer (twos arguments)."""
    return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0


def g_tilde_sq(a: int, b: int, c: int) -> Fraction:
    """Square of the triangle coefficient g~(a,b,c), Eq. A4."""
    return Fraction(fact(a + b - c) * fact(a - b + c) * fact(-a + b + c),
                    fact(a + b + c + 2))


def _signed_sqrt(sign: int, sq: Fraction) -> float:
    return sign * math.sqrt(float(sq)) if sq else 0.0


@lru_cache(maxsize=None)
def sixj_exact(a: int, b: int, c: int, d: int, e: int, f: int):
    """W6j(a,b,c,d,e,f) of Eq. A3 as (sign, value^2) in exact rationals.

    The four triads are (a,b,c), (c,d,e), (a,e,f), (b,d,f); the sum runs over
    n from max(n~1..n~5) to min(n~6..n~8) with n~1=0.
    """
    if not (triangle(a, b, c) and triangle(c, d, e) and triangle(a, e, f)
            and triangle(b, d, f)):
        return 0, Fraction(0)
    n2 = (a + b + c) // 2
    n3 = (c + d + e) // 2
    n4 = (a + e + f) // 2
    n5 = (b + d + f) // 2
    n6 = (a + b + d + e) // 2
    n7 = (a + c + d + f) // 2
    n8 = (b + c + e + f) // 2
    nmin = max(0, n2, n3, n4, n5)
    nmax = min(n6, n7, n8)
    s = Fraction(0)
    for n in range(nmin, nmax + 1):
        den = (math.factorial(n - n2) * math.factorial(n - n3) *
               math.factorial(n - n4) * math.factorial(n - n5) *
               math.factorial(n6 - n) * math.factorial(n7 - n) *
               math.factorial(n8 - n))
        s += Fraction((-1) ** n * math.factorial(n + 1), den)
    pref = g_tilde_sq(a, b, c) * g_tilde_sq(c, d, e) * g_tilde_sq(a, e, f) * g_tilde_sq(b, d, f)
    if s == 0:
        return 0, Fraction(0)
    return (1 if s > 0 else -1), pref * s * s


def sixj(a, b, c, d, e, f) -> float:
    """Wigner 6j {a b c; d e f} (twos arguments), Eq. A3."""
    sg, sq = sixj_exact(a, b, c, d, e, f)
    return _signed_sqrt(sg, sq)


@lru_cache(maxsize=None)
def ninej(j1, j2, j, k1, k2, k, j1p, j2p, jp) -> float:
    """W9j(j1,j2,j,k1,k2,k,j1',j2',j') of Eq. A2 (rows (j1 j2 j), (k1 k2 k),
    (j1' j2' j')), twos arguments.

    x runs in integer steps from max(|j1-j'|, |j2-k|, |k1-j2'|) to
    min(j1+j', j2+k, k1+j2').  The paper prints the lower bound without
    absolute values; a negative x is not a valid spin, so the absolute values
    are taken (the 6j with a violated triangle vanish either way).
    """
    for t in ((j1, j2, j), (k1, k2, k), (j1p, j2p, jp),
              (j1, k1, j1p), (j2, k2, j2p), (j, k, jp)):
        if not triangle(*t):
            return 0.0
    xmin = max(abs(j1 - jp), abs(j2 - k), abs(k1 - j2p))
    xmax = min(j1 + jp, j2 + k, k1 + j2p)
    tot = 0.0
    for x in range(xmin, xmax + 1, 2):
        sign = -1.0 if (x % 2) else 1.0          # (-1)^{2x}
        tot += sign * (x + 1) * (sixj(j1, j2, j, k, jp, x) *
                                 sixj(k1, k2, k, j2, x, j2p) *
                                 sixj(j1p, j2p, jp, x, j1, k1))
    return tot


def ctilde(j1, j2, j, k1, k2, k, j1p, j2p, jp) -> float:
    """Scalar factor C~ of Eq. a (twos arguments).

    Reading: the primed spins label the output (bra) side and the unprimed
    the input (ket) side; reduced matrix elements follow the Clebsch-Gordan
    form of the Wigner-Eckart theorem,
    <j' m'|T^k_q|j m> = <j m; k q | j' m'> <j'||T^k||j>.
    Then <(j1' j2') j'|| [T^{k1} x U^{k2}]^k ||(j1 j2) j> equals
    C~ <j1'||T||j1> <j2'||U||j2>.
    """
    w = ninej(j1, j2, j, k1, k2, k, j1p, j2p, jp)
    if w == 0.0:
        return 0.0
    return math.sqrt((j1p + 1) * (j2p + 1) * (j + 1) * (k + 1)) * w


@lru_cache(maxsize=None)
def cg_exact(j1, m1, j2, m2, J, M):
    """Clebsch-Gordan <j1 m1; j2 m2 | J M> by Racah's closed formula, as
    (sign, value^2).  Independent of the 6j route above."""
    if m1 + m2 != M or not triangle(j1, j2, J):
        return 0, Fraction(0)
    for jj, mm in ((j1, m1), (j2, m2), (J, M)):
        if abs(mm) > jj or (jj + mm) % 2:
            return 0, Fraction(0)
    pref = Fraction((J + 1) * fact(J + j1 - j2) * fact(J - j1 + j2) * fact(j1 + j2 - J),
                    fact(j1 + j2 + J + 2))
    pref *= (fact(J + M) * fact(J - M) * fact(j1 - m1) * fact(j1 + m1) *
             fact(j2 - m2) * fact(j2 + m2))
    s = Fraction(0)
    kmax = (j1 + j2 - J) // 2 + 2 * (j1 + j2 + J)
    for kk in range(0, kmax + 1):
        args = [(j1 + j2 - J) // 2 - kk, (j1 - m1) // 2 - kk, (j2 + m2) // 2 - kk,
                (J - j2 + m1) // 2 + kk, (J - j1 - m2) // 2 + kk]
        if min(args) < 0:
            continue
        den = math.factorial(kk)
        for a in args:
            den *= math.factorial(a)
        s += Fraction((-1) ** kk, den)
    if s == 0:
        return 0, Fraction(0)
    return (1 if s > 0 else -1), pref * s * s


def cg(j1, m1, j2, m2, J, M) -> float:
    """Clebsch-Gordan coefficient (twos arguments, Condon-Shortley phases)."""
    sg, sq = cg_exact(j1, m1, j2, m2, J, M)
    return _signed_sqrt(sg, sq)
