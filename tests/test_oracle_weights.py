"""Pins for the Appendix A weights of the oracle (exact rationals).

Independent derivations: the Gregory end corrections are rebuilt here from the
Gregory difference formula (trapezoid plus forward/backward difference
corrections with the Gregory coefficients), not from Adams-Moulton weights as
the oracle does; BDF weights are the textbook table; every composite rule is
checked for exactness on monomials by brute force.
"""
import os
from fractions import Fraction
from math import comb

import pytest

from oracle import weights as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, den = line.split("/")
        parts = head.split()
        k = int(parts[0])
        out[k] = [Fraction(int(p), int(den)) for p in parts[1:]]
    return out


# Gregory coefficients c_p of the difference corrections (p = 1..5)
GREG_C = [Fraction(1, 12), Fraction(1, 24), Fraction(19, 720), Fraction(3, 160),
          Fraction(863, 60480)]


def gregory_from_differences(k):
    """Left-end weights of int_0^n f = trapezoid + sum_{p=1}^{k} (-1)^{p+1} c_p Delta^p f_0 + (mirror)."""
    w = [Fraction(0)] * (k + 1)
    w[0] = Fraction(1, 2)
    for i in range(1, k + 1):
        w[i] = Fraction(1)
    for p in range(1, k + 1):
        sgn = (-1) ** (p + 1)
        for j in range(p + 1):          # Delta^p f_0 = sum_j (-1)^(p-j) C(p,j) f_j
            w[j] += sgn * GREG_C[p - 1] * (-1) ** (p - j) * comb(p, j)
    return w


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_gregory_golden(k):
    gold = _read_table("gregory_weights.txt")[k]
    assert gregory_from_differences(k) == gold
    assert W.gregory_exact(k) == gold
    assert sum(gold) == Fraction(2 * k + 1, 2)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_bdf_golden(k):
    gold = _read_table("bdf_weights.txt")[k]
    assert W.bdf_exact(k) == gold


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_rules_exact_on_monomials(k):
    for n in range(0, 4 * k + 6):
        w = W.rule_exact(k, n)
        for d in range(k + 1):
            got = sum(wi * Fraction(i) ** d for i, wi in enumerate(w))
            assert got == Fraction(n) ** (d + 1) / (d + 1), (k, n, d)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_polynomial_D_I_exact(k):
    D = W.diff_D_exact(k)
    for m in range(k + 1):
        for d in range(k + 1):
            got = sum(D[m][l] * Fraction(l) ** d for l in range(k + 1))
            want = d * Fraction(m) ** (d - 1) if d > 0 else 0
            assert got == want
        for n in range(k + 1):
            I = W.integ_I_exact(k, m, n)
            for d in range(k + 1):
                got = sum(I[l] * Fraction(l) ** d for l in range(k + 1))
                assert got == (Fraction(n) ** (d + 1) - Fraction(m) ** (d + 1)) / (d + 1)


def test_gregory_interior_is_one_and_symmetric():
    k = 5
    w = W.rule_exact(k, 40)
    assert all(x == 1 for x in w[k + 1:40 - k])
    assert w == w[::-1]
