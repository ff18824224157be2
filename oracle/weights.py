"""Oracle: integration and differentiation weights of Appendix A.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg use it.

Everything here is computed in exact rational arithmetic (``fractions``) and
converted to float at the end, so the weights are the textbook values rather
than the result of a floating-point Vandermonde inversion.

Appendix A (integral and derivative approximations):
  * interpolant P[y_0..y_k](t) = sum_{a,l} h^-a t^a P_al y_l, P = M^-1, M_ja = j^a
  * differentiation D_ml = sum_{a>=1} P_al a m^(a-1)
  * integration I_mnl = sum_a P_al (n^(a+1) - m^(a+1)) / (a+1)
  * backward differentiation a_j = -D_0j
  * Gregory end weights omega_i built from the Adams-Moulton weights.

Reading of the Gregory formula (printed garbled in Appendix A, where the summand
does not depend on the summation index): omega_i = sum_{j=0}^{i} b_j, with b_j
the weights of the (k+1)-step Adams-Moulton method, b_0 multiplying the newest
point.  Equivalently b_j = int_k^{k+1} l_{k+1-j}(x) dx with l the Lagrange basis
on the nodes 0..k+1.  This reproduces the classical Gregory end corrections
(k=2: 3/8, 7/6, 23/24) and sum_i omega_i = k + 1/2.

Reading of the composite rule for k < n < 2k+1 (the paper is silent):
int_0^n = int_0^{n-k} by the order-k polynomial on points 0..k, plus int_{n-k}^{n}
by the same polynomial rule shifted onto points n-k..n.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np


def _inv_rational(M):
    n = len(M)
    A = [[Fraction(x) for x in row] + [Fraction(int(i == j)) for j in range(n)]
         for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [x / piv for x in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return [row[n:] for row in A]


@lru_cache(maxsize=None)
def poly_P(k: int):
    """P = M^-1 with M_ja = j^a, 0 <= j, a <= k (exact)."""
    M = [[Fraction(j) ** a for a in range(k + 1)] for j in range(k + 1)]
    return _inv_rational(M)


@lru_cache(maxsize=None)
def diff_D_exact(k: int):
    """D_ml = sum_{a=1}^k P_al a m^(a-1)."""
    P = poly_P(k)
    return [[sum(P[a][l] * a * Fraction(m) ** (a - 1) for a in range(1, k + 1))
             for l in range(k + 1)] for m in range(k + 1)]


def integ_I_exact(k: int, m, n):
    """I_mnl = sum_{a=0}^k P_al (n^(a+1) - m^(a+1)) / (a+1), l = 0..k."""
    P = poly_P(k)
    m = Fraction(m)
    n = Fraction(n)
    return [sum(P[a][l] * (n ** (a + 1) - m ** (a + 1)) / (a + 1)
                for a in range(k + 1)) for l in range(k + 1)]


@lru_cache(maxsize=None)
def bdf_exact(k: int):
    """a_j = -D_0j."""
    D = diff_D_exact(k)
    return [-D[0][j] for j in range(k + 1)]


def _lagrange_integral(nodes, j, lo, hi):
    """int_lo^hi of the Lagrange basis polynomial of node j (exact)."""
    # build polynomial coefficients of prod_{m != j} (x - x_m)/(x_j - x_m)
    coef = [Fraction(1)]
    den = Fraction(1)
    for m, xm in enumerate(nodes):
        if m == j:
            continue
        den *= (nodes[j] - xm)
        new = [Fraction(0)] * (len(coef) + 1)
        for p, c in enumerate(coef):
            new[p + 1] += c
            new[p] -= c * xm
        coef = new
    lo = Fraction(lo)
    hi = Fraction(hi)
    return sum(c * (hi ** (p + 1) - lo ** (p + 1)) / (p + 1)
               for p, c in enumerate(coef)) / den


@lru_cache(maxsize=None)
def adams_moulton_exact(k: int):
    """Weights b_0..b_{k+1} of the (k+1)-step Adams-Moulton method, b_0 on the
    newest point: b_j = int_k^{k+1} l_{k+1-j}(x) dx, nodes 0..k+1."""
    nodes = [Fraction(i) for i in range(k + 2)]
    return [_lagrange_integral(nodes, k + 1 - j, k, k + 1) for j in range(k + 2)]


@lru_cache(maxsize=None)
def gregory_exact(k: int):
    """omega_i = sum_{j=0}^{i} b_j, i = 0..k."""
    b = adams_moulton_exact(k)
    out = []
    acc = Fraction(0)
    for i in range(k + 1):
        acc += b[i]
        out.append(acc)
    return out


def rule_exact(k: int, n: int):
    """Weights w^(n)_l of int_0^{n} y (unit spacing) as exact rationals.

    n = 0: empty; 1 <= n <= k: I_{0,n,l} on points 0..k (may reach past n);
    k < n < 2k+1: I_{0,n-k,.} on 0..k plus I_{0,k,.} shifted to n-k..n;
    n >= 2k+1: Gregory omega at both ends, 1 inside.
    Returned list has length max(n, k) + 1.
    """
    L = max(n, k) + 1
    w = [Fraction(0)] * L
    if n == 0:
        return w
    if n <= k:
        return list(integ_I_exact(k, 0, n))
    if n < 2 * k + 1:
        for l, x in enumerate(integ_I_exact(k, 0, n - k)):
            w[l] += x
        for l, x in enumerate(integ_I_exact(k, 0, k)):
            w[n - k + l] += x
        return w
    om = gregory_exact(k)
    for l in range(n + 1):
        w[l] = Fraction(1)
    for i in range(k + 1):
        w[i] = om[i]
        w[n - i] = om[i]
    return w


# ---- float views used by the stepper ---------------------------------------

class Weights:
    """Float copies of every weight the scheme uses, for order k."""

    def __init__(self, k: int):
        if not 1 <= k <= 5:
            raise ValueError("integration order k must be in 1..5")
        self.k = k
        self.D = np.array([[float(x) for x in row] for row in diff_D_exact(k)])
        self.a = np.array([float(x) for x in bdf_exact(k)])
        self.omega = np.array([float(x) for x in gregory_exact(k)])
        self._rule = {}
        self._I = {}

    def I(self, m: int, n: int) -> np.ndarray:
        """I_{m,n,l}: weights of int_m^n over the points 0..k (Appendix A)."""
        key = (m, n)
        if key not in self._I:
            self._I[key] = np.array([float(x) for x in integ_I_exact(self.k, m, n)])
        return self._I[key]

    def rule(self, n: int) -> np.ndarray:
        """w^(n)_l of int_0^n (unit spacing): start weights for n <= k, Gregory
        end corrections beyond (Appendix A)."""
        if n not in self._rule:
            self._rule[n] = np.array([float(x) for x in rule_exact(self.k, n)])
        return self._rule[n]

    def extrap(self) -> np.ndarray:
        """Polynomial extrapolation of degree k through the previous k+1 points:
        y_n ~ sum_l e_l y_{n-1-l}, e_l = (-1)^l C(k+1, l+1)."""
        from math import comb
        return np.array([(-1) ** l * comb(self.k + 1, l + 1) for l in range(self.k + 1)],
                        dtype=float)
