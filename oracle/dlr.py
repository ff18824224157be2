"""Oracle: imaginary-time operations on the DLR grid (Sec. 2.5, Tables 4-5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Given the DLR frequencies w_l and nodes tau_i (input data), a function on
(0, beta) is represented as f(tau) = sum_l c_l K(tau, w_l) with the fermionic
Lehmann kernel K(tau, w) = exp(-tau w) / (1 + exp(-beta w)).  The cardinal
functions l_a(tau) = sum_l K(tau, w_l) (K^-1)_{l a} reproduce the values at
the nodes.  Every matrix below is built by evaluating cardinal functions and
integrating them with composite Gauss-Legendre quadrature, refined
geometrically toward the panel ends where exp(-tau w) varies fastest.  The
CUDA library builds the same matrices from closed-form exponential integrals;
the two constructions share nothing.

  e(tau)   evaluation row: f(tau) = e(tau) . f(nodes)          (get_mat_tau)
  Rev      f(beta - tau_i) = Rev . f(nodes)                     (get_*_reversed)
  Q_ab     int_0^beta l_a(tau) l_b(tau) dtau                    (mixed product)
  Phi_aci  int_0^beta l_a(tb) l_c^ext(tb - tau_i) dtb           (Sigma^tv * G^M)
where l^ext(x) = l(x) for x > 0 and xi l(x + beta) for x < 0 ((anti)periodicity
of G^M, Sec. 2.1).
"""
from __future__ import annotations

import numpy as np


def kernel(tau, om, beta):
    """K(tau, w) for arrays tau (n,), om (m,) -> (n, m), overflow-safe.
    The fermionic Lehmann kernel of the DLR (Sec. 2.5)."""
    t = np.asarray(tau, dtype=float)[:, None]
    w = np.asarray(om, dtype=float)[None, :]
    wp = np.where(w >= 0, w, 0.0)
    wn = np.where(w >= 0, 0.0, w)
    kp = np.exp(-t * wp) / (1.0 + np.exp(-beta * wp))
    kn = np.exp((beta - t) * wn) / (1.0 + np.exp(beta * wn))
    return np.where(w >= 0, kp, kn)


def _gl_composite(a, b, levels=24, npts=24):
    """Gauss-Legendre on (a, b), panels geometrically refined toward both
    ends (panel widths halve toward a and toward b)."""
    x, w = np.polynomial.legendre.leggauss(npts)
    mid = 0.5 * (a + b)
    half = 0.5 * (b - a)
    edges = [0.0] + [half * 2.0 ** (-j) for j in range(levels, -1, -1)]
    xs, ws = [], []
    for i in range(len(edges) - 1):
        lo, hi = edges[i], edges[i + 1]
        for s in (1.0, -1.0):  # toward a (s=+1 from a) and toward b (s=-1 from b)
            c = 0.5 * (hi + lo)
            d = 0.5 * (hi - lo)
            pts = c + d * x
            if s > 0:
                xs.append(a + pts)
            else:
                xs.append(b - pts)
            ws.append(d * w)
    xs = np.concatenate(xs)
    ws = np.concatenate(ws)
    assert abs(ws.sum() - (b - a)) < 1e-12 * max(1.0, b - a)
    del mid
    return xs, ws


class DLROracle:
    """Cardinal functions on the DLR nodes and the matrices built from them
    (Sec. 2.5, Tables 4-5): evaluation rows, reversal, product and convolution."""

    def __init__(self, tau_nodes, omega_nodes, beta, xi=-1):
        self.tau = np.asarray(tau_nodes, dtype=float)
        self.om = np.asarray(omega_nodes, dtype=float)
        self.beta = float(beta)
        self.xi = xi
        self.r = len(self.tau)
        self.K = kernel(self.tau, self.om, beta)
        self._lu = None

    def cardinal(self, tau):
        """l_a(tau) for every a: (len(tau), r)."""
        import scipy.linalg as sla
        if self._lu is None:
            self._lu = sla.lu_factor(self.K)
        # l(tau) K = K(tau, .)  ->  K^T l(tau)^T = K(tau, .)^T
        rhs = kernel(np.atleast_1d(tau), self.om, self.beta)
        return sla.lu_solve(self._lu, rhs.T, trans=1).T

    def eval_row(self, tau):
        """e(tau): f(tau) = e(tau) . f(nodes) (Table 4, get_mat_tau)."""
        return self.cardinal(np.atleast_1d(float(tau)))[0]

    def rev(self):
        """Rev: f(beta - tau_i) = Rev . f(nodes) (Table 5, the reversed functions)."""
        return self.cardinal(self.beta - self.tau)

    def Q(self):
        """Q_ab = int_0^beta l_a l_b dtau, the imaginary-time product of the
        mixed terms of Eq. KBEL (Sec. 2.5)."""
        x, w = _gl_composite(0.0, self.beta)
        L = self.cardinal(x)
        return (L * w[:, None]).T @ L

    def phi(self):
        """Phi[a, c, i] = int_0^beta l_a(tb) l_c^ext(tb - tau_i) dtb."""
        r = self.r
        out = np.zeros((r, r, r))
        for i, ti in enumerate(self.tau):
            # tb in (0, ti): argument tb - ti < 0 -> xi * l_c(tb - ti + beta)
            x1, w1 = _gl_composite(0.0, ti)
            x2, w2 = _gl_composite(ti, self.beta)
            La1 = self.cardinal(x1)
            Lc1 = self.xi * self.cardinal(x1 - ti + self.beta)
            La2 = self.cardinal(x2)
            Lc2 = self.cardinal(x2 - ti)
            out[:, :, i] = (La1 * w1[:, None]).T @ Lc1 + (La2 * w2[:, None]).T @ Lc2
        return out

    def conv_tensor(self, gm):
        """W[a, i] = int l_a(tb) G^M_ext(tb - tau_i) dtb as N_o x N_o matrices,
        so that int_0^beta S(tb) G^M(tb - tau_i) dtb = sum_a S(tau_a) W[a, i]."""
        ph = self.phi()
        return np.einsum("aci,cxy->aixy", ph, gm)
