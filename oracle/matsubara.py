"""Oracle: the equilibrium (Matsubara) Dyson equation on the DLR grid
(Eq. KBEM, Sec. 2.5 and 3.2), solved self-consistently.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Representation: G^M(tau) = -sum_l c_l K(tau, w_l) with the DLR frequencies
w_l and K(tau, w) = e^{-tau w}/(1 + e^{-beta w}); its Fourier series is
G(i nu) = sum_l c_l / (i nu - w_l), nu = (2n+1) pi / beta.  The Dyson
equation G(i nu) = [i nu - eps - Sigma(i nu)]^{-1} is imposed on r
fermionic frequencies picked from |n| <= n_max by column-pivoted QR of the
matrix [1/(i nu_n - w_l)] (scipy), so that values at those frequencies
determine the coefficients.  Sigma^M(tau) on the tau nodes from G^M, for the
contour functionals of the real-time models restricted to the imaginary
branch (G^M = -i G(-i tau, 0), Table 1):
  bethe       Sigma = v^2 G
  nambu       Delta = v^2 sigma_z G sigma_z  +  second Born
              Sigma_ij = -U^2 [G_ij G_{bi bj} - G_{bi j} G_{i bj}](tau) G_{bj bi}(-tau)
              +  Holstein  g^2 [(n_B+1) e^{-w0 tau} + n_B e^{w0 tau}] sigma_z G sigma_z
              (G(-tau) = xi G(beta - tau)); the Fock term -U rho_ij [i = bar j]
              with rho = -G^M(beta^-) shifts eps
  lattice2b   Sigma_r(tau) = -U^2 G_r(tau)^2 G_{-r}(-tau), G_r = (1/N_k) sum_k e^{ikr} G_k
A pairing field eta (eps_01 = eps_10 += eta) can be applied for the first
n_eta iterations (Sec. 4.1: symmetry breaking in the Matsubara iterations).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dlr import DLROracle, kernel


def matsubara_nodes(om, beta, n_max):
    """r fermionic Matsubara frequencies nu_n, |n| <= n_max, picked by
    column-pivoted QR of [1/(i nu_n - w_l)], where the Dyson equation is
    imposed (Sec. 2.5)."""
    n = np.arange(-n_max, n_max)
    nu = (2 * n + 1) * np.pi / beta
    A = 1.0 / (1j * nu[:, None] - np.asarray(om)[None, :])
    _, _, piv = sla.qr(A.T, pivoting=True, mode="economic")
    return np.sort(nu[piv[:len(om)]])


class MatsubaraOracle:
    """Self-consistent equilibrium Dyson equation (Eq. KBEM) on the DLR grid."""

    def __init__(self, tau, om, beta, xi=-1, n_max=None):
        self.tau = np.asarray(tau, float)
        self.om = np.asarray(om, float)
        self.beta = float(beta)
        self.xi = xi
        self.r = len(self.tau)
        self.Kt = kernel(self.tau, self.om, beta)                     # (r, r)
        if n_max is None:
            n_max = int(2 * beta * np.abs(self.om).max() / (2 * np.pi)) + 100
        self.nu = matsubara_nodes(self.om, beta, n_max)
        self.Kn = 1.0 / (1j * self.nu[:, None] - self.om[None, :])    # (r, r)
        self.rev = DLROracle(self.tau, self.om, beta, xi).rev()
        self.ebeta = DLROracle(self.tau, self.om, beta, xi).eval_row(beta)

    def to_freq(self, g):
        """values on tau nodes (r, ...) -> values at the Matsubara nodes."""
        c = np.linalg.solve(self.Kt, -g.reshape(self.r, -1))
        return (self.Kn @ c).reshape(g.shape)

    def to_tau(self, gn):
        """values at the Matsubara nodes -> values on the tau nodes (inverse of to_freq)."""
        c = np.linalg.solve(self.Kn, gn.reshape(self.r, -1))
        return (-(self.Kt @ c)).reshape(gn.shape).real if np.isrealobj(gn) else (-(self.Kt @ c)).reshape(gn.shape)

    def reversed(self, g):
        """g(beta - tau_i) on the nodes."""
        return np.einsum("ij,j...->i...", self.rev, g)

    def dyson(self, eps, sig_tau):
        """eps (N, No, No) per instance, sig_tau (N, r, No, No) -> G^M (N, r, No, No)."""
        N, No = eps.shape[0], eps.shape[-1]
        out = np.zeros((N, self.r, No, No), complex)
        for n in range(N):
            sn = self.to_freq(sig_tau[n])
            gn = np.array([np.linalg.inv(1j * nu * np.eye(No) - eps[n] - sn[i]) for i, nu in enumerate(self.nu)])
            out[n] = self.to_tau(gn)
        return out

    def sigma(self, model, G, params):
        """Sigma^M(tau) on the nodes for the functionals listed in the module
        header (Eq. Hybrid, Eq. Sigma2B, Migdal, lattice second Born)."""
        N, r, No, _ = G.shape
        S = np.zeros_like(G)
        if model == "bethe":
            return params["v"] ** 2 * G
        if model == "nambu":
            v, U = params.get("v", 1.0), params.get("U", 0.0)
            g, w0 = params.get("g", 0.0), params.get("w0", 1.0)
            s = np.array([1.0, -1.0])
            ss = np.outer(s, s)
            S = v * v * ss * G
            if U:
                Gm = self.xi * np.array([self.reversed(G[n]) for n in range(N)])   # G(-tau)
                for i in range(2):
                    for j in range(2):
                        bi, bj = 1 - i, 1 - j
                        S[..., i, j] += -U * U * (G[..., i, j] * G[..., bi, bj] - G[..., bi, j] * G[..., i, bj]) \
                            * Gm[..., bj, bi]
            if g:
                nb = 1.0 / np.expm1(self.beta * w0)
                d = (nb + 1) * np.exp(-w0 * self.tau) + nb * np.exp(w0 * self.tau)
                S += g * g * d[None, :, None, None] * ss * G
            return S
        if model == "lattice2b":
            L, U = params["L"], params["U"]
            g = G[..., 0, 0].reshape(L, L, r)
            gm = self.xi * np.array([self.reversed(G[n, :, 0, 0]) for n in range(N)]).reshape(L, L, r)
            gr = np.fft.ifft2(g, axes=(0, 1))
            gmr = np.fft.fft2(gm, axes=(0, 1)) / (L * L)       # G_{-r}(-tau)
            sk = np.fft.fft2(-U * U * gr ** 2 * gmr, axes=(0, 1)).reshape(N, r)
            S[..., 0, 0] = sk
            return S
        raise ValueError(model)

    def solve(self, model, eps, params, G0=None, tol=1e-12, max_iter=500, mix=0.5, eta=0.0, n_eta=0):
        """Self-consistent G^M (N, r, No, No) and the equilibrium eps with the
        Fock shift (Nambu).  eps: (N, No, No) equilibrium-branch levels."""
        eps = np.asarray(eps, complex)
        N, No = eps.shape[0], eps.shape[-1]
        G = np.zeros((N, self.r, No, No), complex) if G0 is None else np.array(G0, complex)
        if G0 is None:
            G = self.dyson(eps, G)
        e_eff = eps.copy()
        for it in range(1, max_iter + 1):
            e_eff = eps.copy()
            if model == "nambu":
                U = params.get("U", 0.0)
                rho = -np.einsum("c,nc...->n...", self.ebeta, G)
                e_eff[:, 0, 1] += -U * rho[:, 0, 1]
                e_eff[:, 1, 0] += -U * rho[:, 1, 0]
                if it <= n_eta:
                    e_eff[:, 0, 1] += eta
                    e_eff[:, 1, 0] += eta
            Gn = self.dyson(e_eff, self.sigma(model, G, params))
            err = np.abs(Gn - G).max()
            G = mix * Gn + (1 - mix) * G if it > 1 else Gn
            if err < tol and it > n_eta:
                G = Gn
                break
        return G, e_eff, it, err
