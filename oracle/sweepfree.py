"""Oracle: the sweep-free variant of the time step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is not the paper's discretisation but a variant of it: every point of
the new retarded row and of the new lesser column is
an independent small solve or a quadrature over stored history, so nothing is
solved point after point along the row.  It shares the bootstrap (the k + 1
start steps), the mixed component (Eq. KBET), the lesser source q (Eq. KBEL,
second and third terms) and every weight with the paper's scheme
(``oracle/kbe.py``); it differs from it at O(h^k).

Retarded row T.  The k points next to the diagonal, t' = T - 1 .. T - k, are
the start block of Eq. KBER, solved together as in the paper's scheme (a fixed
k N_o x k N_o system, not a sweep).  Every t' = T - n with n > k comes from the
retarded Dyson equation in its FIRST time argument,
i d_t G^R(t,t') = eps(t) G^R(t,t') + int_{t'}^{t} Sigma^R(t,s) G^R(s,t') ds,
taken at t = T with the BDF derivative over the rows T - j, on its own:

    (i/h) sum_j a_j G^R(T-j, t') = eps(T) G^R(T,t') + h sum_{l=0}^{n} w^(n)_l Sigma^R(T, t'+l) G^R(t'+l, t')

with the rule w^(n) of Appendix A (every point it uses lies in [t', T] because
n > k).  The unknown G^R(T, t') enters through a_0 and the l = n term: one
N_o x N_o solve per t'.  G^R(T, T) = -i.  (Reading: a start for n <= k from the
left equation itself, with the BDF stencil continued across the diagonal by
G^R_x(a, b) = -[G^R(b, a)]^dagger, was tried first and is unstable, its error
growing about twofold per step next to the diagonal; the start block is kept.)

Lesser column T.  The lesser equation of Eq. KBEL in its first argument is a
linear Volterra integro-differential equation for x(t) = G^<(t, T) whose
resolvent is G^R, so (a Duhamel / Keldysh form)

    x(t) = i G^R(t, 0) x(0) + int_0^t G^R(t, s) q(s) ds,   x(0) = -[G^tv(T, 0+)]^dagger,

discretised with w^(t) (Gregory; for t < k the start weights I_{0,t,l} on the
points 0..k, above the diagonal through G^R_x):

    x_t = i G^R(t, 0) x_0 + h sum_l w^(t)_l G^R_x(t, l) q_l,   t = 1..T

(t = T - 1 at most with the diagonal density-matrix scheme, which then gives
x_T as in the paper's scheme).
"""
from __future__ import annotations

import numpy as np

from .kbe import KBEOracle, _dag


class SweepFreeOracle(KBEOracle):
    """The dense FP64 stepper of the sweep-free variant (module docstring);
    everything but the retarded row and the lesser column is inherited."""

    def gR_x(self, a, b):
        """G^R(a, b), continued above the diagonal."""
        return self.GR[a, b] if a >= b else -_dag(self.GR[b, a])

    def solve_ret(self, T):
        """Row G^R(T, .): the start block for t' = T-1..T-k, then one
        independent solve per t' from the first-argument equation (module
        docstring)."""
        k, h, W = self.k, self.h, self.W
        a = W.a
        y = self._ret_start_block(T)
        for s in range(k + 1):
            self.GR[T, T - s] = y[s]
        M = (1j * a[0] / h) * self.I1 - self.ep(T)
        for n in range(k + 1, T + 1):
            tp = T - n
            w = W.rule(n)
            rhs = -(1j / h) * sum(a[j] * self.GR[T - j, tp] for j in range(1, k + 1))
            for l in range(n):
                rhs = rhs + h * w[l] * (self.SR[T, tp + l] @ self.GR[tp + l, tp])
            self.GR[T, tp] = np.linalg.solve(M - h * w[n] * self.SR[T, T], rhs)

    def solve_les(self, T):
        """Column G^<(., T) from its resolvent (Duhamel) form with the lesser
        source q; x_T from the density-matrix scheme when rho_mode = 1."""
        k, h, W, No = self.k, self.h, self.W, self.no
        q = self.lesser_source(T)
        x = np.zeros((T + 1, No, No), complex)
        x[0] = -_dag(self.gtv_at0(T))
        last = T if self.rho_mode == 0 else T - 1
        for t in range(1, last + 1):
            w = W.rule(t)                       # max(t, k) + 1 weights
            acc = 1j * (self.GR[t, 0] @ x[0])
            for l in range(len(w)):
                acc = acc + h * w[l] * (self.gR_x(t, l) @ q[l])
            x[t] = acc
        if self.rho_mode == 1:
            x[T] = self._rho_diagonal(T, x, q)
        self.GLs[T, :T + 1] = x
