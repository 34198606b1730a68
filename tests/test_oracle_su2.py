"""Pins for the oracle's Clebsch-Gordan and 6-j routines (Racah formulas).

Independent references: coupled states built by the lowering operator J- and
Gram-Schmidt on product states (Condon-Shortley phase: <j1 j1 j2 (J-j1)|J J> > 0),
and the recoupling overlap that defines the 6-j symbol."""
import itertools

import numpy as np
import pytest

from oracle.su2 import cg, sixj


def jminus(tj):
    """Matrix of J- on |j m>, m = j..-j (index 0 = m=j)."""
    j = tj / 2
    ms = [j - k for k in range(tj + 1)]
    M = np.zeros((tj + 1, tj + 1))
    for a, m in enumerate(ms[:-1]):
        M[a + 1, a] = np.sqrt(j * (j + 1) - m * (m - 1))
    return M


def ladder_cg(tj1, tj2):
    """All coupled states |J M> in the product basis by J- and Gram-Schmidt."""
    d1, d2 = tj1 + 1, tj2 + 1
    Jm = np.kron(jminus(tj1), np.eye(d2)) + np.kron(np.eye(d1), jminus(tj2))
    states = {}
    found = []
    for tJ in range(tj1 + tj2, abs(tj1 - tj2) - 1, -2):
        # highest weight M = J: product states with m1 + m2 = J
        tM = tJ
        basis = []
        for a in range(d1):
            for b in range(d2):
                if (tj1 - 2 * a) + (tj2 - 2 * b) == tM:
                    e = np.zeros(d1 * d2); e[a * d2 + b] = 1.0
                    basis.append(e)
        B = np.array(basis).T
        v = B @ np.linalg.lstsq(B, np.ones(d1 * d2) * 0, rcond=None)[0]
        # pick the vector in span(B) orthogonal to all found states with this M
        P = B.copy()
        for f in found:
            if abs(f[1] - tM) == 0:
                P = P - np.outer(f[2], f[2] @ P)
        u, s, _ = np.linalg.svd(P)
        v = u[:, 0]
        # Condon-Shortley: coefficient of m1 = j1 positive
        a = 0
        b = (tj2 - (tM - tj1)) // 2
        if v[a * d2 + b] < 0:
            v = -v
        cur = v
        for k in range(tJ + 1):
            tMk = tJ - 2 * k
            states[(tJ, tMk)] = cur
            found.append((tJ, tMk, cur))
            if k < tJ:
                nxt = Jm @ cur
                cur = nxt / np.linalg.norm(nxt)
    return states


@pytest.mark.parametrize("tj1,tj2", [(1, 1), (2, 1), (2, 2), (3, 1), (4, 3), (5, 2)])
def test_cg_matches_ladder_construction(tj1, tj2):
    states = ladder_cg(tj1, tj2)
    d2 = tj2 + 1
    for (tJ, tM), v in states.items():
        for a in range(tj1 + 1):
            for b in range(tj2 + 1):
                tm1, tm2 = tj1 - 2 * a, tj2 - 2 * b
                assert abs(cg(tj1, tm1, tj2, tm2, tJ, tM) - v[a * d2 + b]) < 1e-12


def recoupling_overlap(t1, t2, t3, t12, t23, tJ):
    """<(j1 j2)j12, j3; J M=J | j1, (j2 j3)j23; J M=J> from CG sums."""
    tot = 0.0
    tM = tJ
    for tm1 in range(-t1, t1 + 1, 2):
        for tm2 in range(-t2, t2 + 1, 2):
            tm3 = tM - tm1 - tm2
            if abs(tm3) > t3:
                continue
            a = cg(t1, tm1, t2, tm2, t12, tm1 + tm2) * cg(t12, tm1 + tm2, t3, tm3, tJ, tM)
            b = cg(t2, tm2, t3, tm3, t23, tm2 + tm3) * cg(t1, tm1, t23, tm2 + tm3, tJ, tM)
            tot += a * b
    return tot


@pytest.mark.parametrize("t1,t2,t3,tJ", [(1, 1, 1, 1), (2, 1, 1, 2), (3, 1, 1, 1), (4, 1, 1, 4),
                                        (2, 1, 1, 0), (5, 1, 1, 3), (1, 1, 0, 0)])
def test_sixj_is_the_recoupling_coefficient(t1, t2, t3, tJ):
    for t12 in range(abs(t1 - t2), t1 + t2 + 1, 2):
        for t23 in range(abs(t2 - t3), t2 + t3 + 1, 2):
            ov = recoupling_overlap(t1, t2, t3, t12, t23, tJ)
            ph = (-1) ** ((t1 + t2 + t3 + tJ) // 2)
            val = ph * np.sqrt((t12 + 1) * (t23 + 1)) * sixj(t1, t2, t12, t3, tJ, t23)
            assert abs(ov - val) < 1e-12


def test_sixj_orthogonality_and_special_value():
    for a, b, c, d in itertools.product(range(0, 5), repeat=4):
        fs = range(0, 10)
        for f in fs:
            for fp in fs:
                s = sum((x + 1) * (f + 1) * sixj(a, b, x, c, d, f) * sixj(a, b, x, c, d, fp)
                        for x in range(0, 10))
                want = 1.0 if (f == fp and _tri(a, d, f) and _tri(b, c, f)) else 0.0
                assert abs(s - want) < 1e-11
    # {a b c; 0 c b} = (-1)^(a+b+c) / sqrt((2b+1)(2c+1))
    for a, b, c in itertools.product(range(0, 6), repeat=3):
        if _tri(a, b, c):
            want = (-1) ** ((a + b + c) // 2) / np.sqrt((b + 1) * (c + 1))
            assert abs(sixj(a, b, c, 0, c, b) - want) < 1e-13


def _tri(a, b, c):
    return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0
