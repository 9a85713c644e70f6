"""Pins of the oracle's 6j (Eq. A3), 9j (Eq. A2) and C~ (Eq. a).

Each check is fixed by the mathematics, not by retyping the formula: closed
forms, orthogonality, the symmetry groups, and brute-force recoupling
overlaps computed from Clebsch-Gordan sums (which do not use the 6j code).
All spins are twos integers.
"""
import itertools
import math

import pytest

from oracle import su2


def spins(maxtwo):
    return range(0, maxtwo + 1)


def test_sixj_closed_form_zero_entry():
    # {a b c; 0 c b} = (-1)^{a+b+c} / sqrt((2b+1)(2c+1))
    for a, b, c in itertools.product(spins(6), repeat=3):
        if not su2.triangle(a, b, c):
            continue
        want = (-1) ** ((a + b + c) // 2) / math.sqrt((b + 1) * (c + 1))
        assert su2.sixj(a, b, c, 0, c, b) == pytest.approx(want, abs=1e-14)


def test_sixj_known_values():
    # {1/2 1/2 1; 1/2 1/2 1} = 1/6 and {1 1 1; 1 1 1} = 1/6
    assert su2.sixj(1, 1, 2, 1, 1, 2) == pytest.approx(1 / 6, abs=1e-15)
    assert su2.sixj(2, 2, 2, 2, 2, 2) == pytest.approx(1 / 6, abs=1e-15)
    # {1/2 1/2 0; 1/2 1/2 1} = 1/2 ; {1/2 1/2 1; 1/2 1/2 0} = 1/2
    assert su2.sixj(1, 1, 0, 1, 1, 2) == pytest.approx(0.5, abs=1e-15)


def test_sixj_orthogonality():
    # sum_x (2x+1)(2f+1) {a b x; c d f}{a b x; c d f'} = delta_{ff'} when the
    # triads (a, d, f) and (c, b, f) are allowed (Edmonds 6.2.9)
    for a, b, c, d in itertools.product(spins(4), repeat=4):
        for f in range(0, 9):
            for fp in range(0, 9):
                s = 0.0
                for x in range(0, 13):
                    s += (x + 1) * (f + 1) * su2.sixj(a, b, x, c, d, f) * su2.sixj(a, b, x, c, d, fp)
                valid = f == fp and su2.triangle(a, d, f) and su2.triangle(c, b, f)
                assert s == pytest.approx(1.0 if valid else 0.0, abs=1e-12)


def test_sixj_tetrahedral_symmetry():
    for a, b, c, d, e, f in itertools.product(range(0, 5), repeat=6):
        v = su2.sixj(a, b, c, d, e, f)
        cols = [(a, d), (b, e), (c, f)]
        for perm in itertools.permutations(range(3)):
            p = [cols[i] for i in perm]
            for flip in ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)):
                q = [(y, x) if fl else (x, y) for (x, y), fl in zip(p, flip)]
                w = su2.sixj(q[0][0], q[1][0], q[2][0], q[0][1], q[1][1], q[2][1])
                assert w == pytest.approx(v, abs=1e-14)


def _recoupling_6j(j1, j2, j12, j3, J, j23):
    """<(j1 j2) j12, j3; J M | j1, (j2 j3) j23; J M> from CG sums, M = J."""
    M = J
    s = 0.0
    for m1 in range(-j1, j1 + 1, 2):
        for m2 in range(-j2, j2 + 1, 2):
            m3 = M - m1 - m2
            if abs(m3) > j3:
                continue
            s += (su2.cg(j1, m1, j2, m2, j12, m1 + m2) * su2.cg(j12, m1 + m2, j3, m3, J, M) *
                  su2.cg(j2, m2, j3, m3, j23, m2 + m3) * su2.cg(j1, m1, j23, m2 + m3, J, M))
    return s


def test_sixj_against_cg_recoupling():
    n = 0
    for j1, j2, j3 in itertools.product(range(0, 4), repeat=3):
        for j12 in range(abs(j1 - j2), j1 + j2 + 1, 2):
            for j23 in range(abs(j2 - j3), j2 + j3 + 1, 2):
                for J in range(abs(j12 - j3), j12 + j3 + 1, 2):
                    if not su2.triangle(j1, j23, J):
                        continue
                    ov = _recoupling_6j(j1, j2, j12, j3, J, j23)
                    sign = (-1) ** ((j1 + j2 + j3 + J) // 2)
                    want = sign * math.sqrt((j12 + 1) * (j23 + 1)) * su2.sixj(j1, j2, j12, j3, J, j23)
                    assert ov == pytest.approx(want, abs=1e-13)
                    n += 1
    assert n > 100


def _recoupling_9j(j1, j2, j12, j3, j4, j34, j13, j24, J):
    """<(j1 j2)j12,(j3 j4)j34; J M | (j1 j3)j13,(j2 j4)j24; J M>, M = J."""
    M = J
    s = 0.0
    for m1 in range(-j1, j1 + 1, 2):
        for m2 in range(-j2, j2 + 1, 2):
            for m3 in range(-j3, j3 + 1, 2):
                m4 = M - m1 - m2 - m3
                if abs(m4) > j4:
                    continue
                a = su2.cg(j1, m1, j2, m2, j12, m1 + m2) * su2.cg(j3, m3, j4, m4, j34, m3 + m4) * \
                    su2.cg(j12, m1 + m2, j34, m3 + m4, J, M)
                if a == 0.0:
                    continue
                b = su2.cg(j1, m1, j3, m3, j13, m1 + m3) * su2.cg(j2, m2, j4, m4, j24, m2 + m4) * \
                    su2.cg(j13, m1 + m3, j24, m2 + m4, J, M)
                s += a * b
    return s


def test_ninej_against_cg_recoupling():
    n = 0
    for j1, j2, j3, j4 in itertools.product(range(0, 3), repeat=4):
        for j12 in range(abs(j1 - j2), j1 + j2 + 1, 2):
            for j34 in range(abs(j3 - j4), j3 + j4 + 1, 2):
                for j13 in range(abs(j1 - j3), j1 + j3 + 1, 2):
                    for j24 in range(abs(j2 - j4), j2 + j4 + 1, 2):
                        for J in range(abs(j12 - j34), j12 + j34 + 1, 2):
                            if not su2.triangle(j13, j24, J):
                                continue
                            ov = _recoupling_9j(j1, j2, j12, j3, j4, j34, j13, j24, J)
                            want = math.sqrt((j12 + 1) * (j34 + 1) * (j13 + 1) * (j24 + 1)) * \
                                su2.ninej(j1, j2, j12, j3, j4, j34, j13, j24, J)
                            assert ov == pytest.approx(want, abs=1e-13)
                            n += 1
    assert n > 200


def test_ninej_zero_entry_reduction():
    # {a b e; c d e; f f 0} = (-1)^{b+c+e+f} / sqrt((2e+1)(2f+1)) {a b e; d c f}
    for a, b, c, d in itertools.product(range(0, 4), repeat=4):
        for e in range(0, 7):
            for f in range(0, 7):
                v = su2.ninej(a, b, e, c, d, e, f, f, 0)
                sign = (-1) ** ((b + c + e + f) // 2) if (b + c + e + f) % 2 == 0 else 0
                want = sign / math.sqrt((e + 1) * (f + 1)) * su2.sixj(a, b, e, d, c, f) if sign else 0.0
                assert v == pytest.approx(want, abs=1e-14)


def test_ninej_symmetries():
    import random
    rng = random.Random(3)
    for _ in range(300):
        m = [[rng.randrange(0, 4) for _ in range(3)] for _ in range(3)]
        v = su2.ninej(*m[0], *m[1], *m[2])
        tot = sum(sum(r) for r in m)
        t = [list(x) for x in zip(*m)]
        assert su2.ninej(*t[0], *t[1], *t[2]) == pytest.approx(v, abs=1e-14)
        for perm in itertools.permutations(range(3)):
            odd = sum(1 for i in range(3) for j in range(i + 1, 3) if perm[i] > perm[j]) % 2
            sg = (-1) ** (tot // 2) if (odd and tot % 2 == 0) else (1 if not odd else None)
            r = [m[i] for i in perm]
            c = [[row[i] for i in perm] for row in m]
            if sg is None:
                continue
            assert su2.ninej(*r[0], *r[1], *r[2]) == pytest.approx(sg * v, abs=1e-14)
            assert su2.ninej(*c[0], *c[1], *c[2]) == pytest.approx(sg * v, abs=1e-14)


def test_ctilde_scalar_is_one():
    for j1, j2 in itertools.product(range(0, 6), repeat=2):
        for j in range(abs(j1 - j2), j1 + j2 + 1, 2):
            assert su2.ctilde(j1, j2, j, 0, 0, 0, j1, j2, j) == pytest.approx(1.0, abs=2e-15)


def test_ctilde_h_factor_reduces_to_6j():
    # k=0 overall: C~(j1,j2,S;k,k,0;j1',j2',S) = (-1)^{j1'+j2+S+k}
    #   sqrt((2j1'+1)(2j2'+1)/(2k+1)) {j1' j2' S; j2 j1 k} ... checked against
    # the zero-entry 9j reduction to the 6j, with the prefactor of Eq. a.
    for j1, j2, k in itertools.product(range(0, 5), repeat=3):
        for S in range(abs(j1 - j2), j1 + j2 + 1, 2):
            for j1p in range(abs(j1 - k), j1 + k + 1, 2):
                for j2p in range(abs(j2 - k), j2 + k + 1, 2):
                    if not su2.triangle(j1p, j2p, S):
                        continue
                    c = su2.ctilde(j1, j2, S, k, k, 0, j1p, j2p, S)
                    # 9j {j1 j2 S; k k 0; j1' j2' S} -> transpose {j1 k j1'; j2 k j2'; S 0 S}
                    # zero-entry form {a b e; c d e; f f 0} after moving the 0 to the corner:
                    nj = su2.ninej(j1, k, j1p, j2, k, j2p, S, 0, S)
                    want = math.sqrt((j1p + 1) * (j2p + 1) * (S + 1) * (0 + 1)) * nj
                    assert c == pytest.approx(want, abs=1e-14)
                    # and it is non-zero only through a single 6j
                    six = su2.sixj(j1, j2, S, j2p, j1p, k)
                    assert (abs(c) > 1e-14) == (abs(six) > 1e-14)
