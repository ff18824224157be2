"""Oracle: 2D Hubbard lattice in the second-Born approximation (Sec. 4.2),
one uncompressed FP64 KBE oracle per k-point, stepped in lockstep because
the self-energy couples all k.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sigma is the paramagnetic second-Born bubble evaluated in real space
(Sec. 4.2, the FFT route): with
    X_r = (1/N_k) sum_k e^{i k.r} X_k          (numpy ifft2)
    Y_{-r} = (1/N_k) sum_k e^{-i k.r} Y_k       (numpy fft2 / N_k)
the lesser and greater components of the current row are
    Sigma^>_r(T, t) = U(T) U(t) G^>_r(T, t)^2 G^<_{-r}(t, T),
    Sigma^<_r(T, t) = U(T) U(t) G^<_r(T, t)^2 G^>_{-r}(t, T),
transformed back with Sigma_k = sum_r e^{-i k.r} Sigma_r (numpy fft2);
Sigma^R_k = Sigma^>_k - Sigma^<_k for t <= T.  The mixed part takes the
imaginary branch latest on the contour:
    Sigma^tv_r(T, tau) = U(T) U(0_|) G^tv_r(T, tau)^2 G^vt_{-r}(tau, T).
k-points are k = 2 pi (m_x, m_y) / L, instance n = m_x L + m_y.
"""
from __future__ import annotations

import numpy as np

from .kbe import KBEOracle
from .models import Model


class _Slave(Model):
    """Per-k placeholder: the coupled driver fills Sigma for every k."""
    name = "lattice_k"
    self_consistent = True

    def eval_step(self, st, T):
        pass


def lattice_sigma(orcs, L, U, T):
    """Fill Sigma^R(T, t), Sigma^<(t, T) (t <= T) and Sigma^tv(T, tau) of every
    k-point oracle from their current rows."""
    nk = L * L
    n = T + 1

    def grid(a):                                    # (nk, ...) -> (L, L, ...)
        return a.reshape((L, L) + a.shape[1:])

    GR = np.array([o.GR[T, :n, 0, 0] for o in orcs])          # (nk, n)
    GLc = np.array([o.GLs[T, :n, 0, 0] for o in orcs])        # G^<(t, T)
    GLr = -np.conj(GLc)                                        # G^<(T, t)
    GGr = GR + GLr                                             # G^>(T, t)
    GGc = -np.conj(GGr)                                        # G^>(t, T)
    uu = U[T + 1] * U[1:T + 2]

    def to_r(x):
        return np.fft.ifft2(grid(x), axes=(0, 1))
    def to_mr(y):
        return np.fft.fft2(grid(y), axes=(0, 1)) / nk
    def to_k(s):
        return np.fft.fft2(s, axes=(0, 1)).reshape((nk,) + s.shape[2:])
    Sg = to_k(uu * to_r(GGr) ** 2 * to_mr(GLc))
    Sl = to_k(uu * to_r(GLr) ** 2 * to_mr(GGc))
    gtv = np.array([o.GTV[T, :, 0, 0] for o in orcs])          # (nk, r)
    gvt = np.array([o.gvt(T)[:, 0, 0] for o in orcs])          # G^vt(tau_i, T)
    Stv = to_k(U[T + 1] * U[0] * to_r(gtv) ** 2 * to_mr(gvt))
    for q, o in enumerate(orcs):
        o.SR[T, :n, 0, 0] = Sg[q] - Sl[q]
        o.SLs[T, :n, 0, 0] = -np.conj(Sl[q])
        o.STV[T, :, 0, 0] = Stv[q]


class LatticeOracle:
    """N_k = L^2 coupled single-orbital oracles (one per k-point)."""

    def __init__(self, L, nt, h, k, beta, eps, gm, tau, omega, U, rho_mode=0, tol=1e-12, max_iter=50):
        self.L = int(L)
        self.U = np.asarray(U, dtype=float)
        self.tol = float(tol)
        self.max_iter = int(max_iter)
        self.orcs = [KBEOracle(nt, h, k, beta, eps[q], gm[q], tau, omega, _Slave(), rho_mode=rho_mode,
                               tol=tol, max_iter=max_iter) for q in range(self.L ** 2)]
        self.k = int(k)
        self.nt = int(nt)

    def bootstrap(self):
        """Start square of every k-point, iterated together with the shared
        Sigma (Sec. 3.3 applied to the coupled lattice of Sec. 4.2)."""
        k = self.k
        for o in self.orcs:
            o.hf_guess()
        for it in range(1, 200 + 1):
            old = [(o.GR[:k + 1, :k + 1].copy(), o.GLs[:k + 1, :k + 1].copy(), o.GTV[:k + 1].copy())
                   for o in self.orcs]
            for t in range(k + 1):
                lattice_sigma(self.orcs, self.L, self.U, t)
            for o in self.orcs:
                o._boot_mixed()
                o._boot_ret()
                o._boot_les()
            err = max(max(np.abs(o.GR[:k + 1, :k + 1] - a).max(), np.abs(o.GLs[:k + 1, :k + 1] - b).max(),
                          np.abs(o.GTV[:k + 1] - c).max()) for o, (a, b, c) in zip(self.orcs, old))
            if err < self.tol:
                break
        for t in range(k + 1):
            lattice_sigma(self.orcs, self.L, self.U, t)

    def step(self, T):
        """Time step T of every k-point, all iterated together until the
        largest change over k is below tol (Sec. 3.4, Sec. 4.2)."""
        for o in self.orcs:
            o.extrapolate(T)
        for it in range(1, self.max_iter + 1):
            old = [(o.GR[T, :T + 1].copy(), o.GLs[T, :T + 1].copy(), o.GTV[T].copy()) for o in self.orcs]
            lattice_sigma(self.orcs, self.L, self.U, T)
            for o in self.orcs:
                o.solve_ret(T)
                o.solve_mixed(T)
                o.solve_les(T)
            err = max(max(np.abs(o.GR[T, :T + 1] - a).max(), np.abs(o.GLs[T, :T + 1] - b).max(),
                          np.abs(o.GTV[T] - c).max()) for o, (a, b, c) in zip(self.orcs, old))
            if err < self.tol:
                break

    def run(self):
        """Bootstrap and step to nt - 1."""
        self.bootstrap()
        for T in range(self.k + 1, self.nt):
            self.step(T)
        return self

    def observables(self, A):
        """Per time t: n = -(i/N_k) sum_k G^<_k(t,t), E_kin = -(2i/N_k) sum_k
        eps_k G^<_k(t,t) with eps_k = -2(cos k_x + cos k_y), and the current
        j = -(2i/N_k) sum_k v^x_{k-A(t)} G^<_k(t,t), v^x_k = 2 sin k_x
        (Sec. 4.2, the factor 2 is the spin sum)."""
        L = self.L
        m = np.arange(L) * 2 * np.pi / L
        kx = np.repeat(m, L)
        ky = np.tile(m, L)
        ek = -2 * (np.cos(kx) + np.cos(ky))
        gl = np.array([[o.GLs[t, t, 0, 0] for t in range(self.nt)] for o in self.orcs])   # (nk, nt)
        nk = L * L
        n = (-1j / nk * gl.sum(0)).real
        ekin = (-2j / nk * (ek[:, None] * gl).sum(0)).real
        vx = 2 * np.sin(kx[:, None] - np.asarray(A)[None, 1:self.nt + 1])
        j = (-2j / nk * (vx * gl).sum(0)).real
        return n, ekin, j

    def interaction_energy(self):
        """Correlation part of the interaction energy per site for t > k (NaN
        for t <= k, where the start rules reach past t) (Galitskii-Migdal on
        the contour, spin summed):
            E_int(t) = -(i/N_k) sum_k (Sigma_k * G_k)^<(t, t),
            (Sigma * G)^<(t, t) = int_0^t [Sigma^R(t,s) G^<(s,t) + Sigma^<(t,s) G^A(s,t)] ds
                                  - i int_0^beta Sigma^tv(t,tau) G^vt(tau,t) dtau,
        the time integrals with the scheme's rule w^(t) (Appendix A), the
        imaginary-time one with the DLR product weights Q (zero after a quench
        from U = 0, where Sigma^tv vanishes)."""
        nk = len(self.orcs)
        out = np.full(self.nt, np.nan)
        for t in range(self.k + 1, self.nt):
            acc = 0.0
            for o in self.orcs:
                wt = o.W.rule(t)[:t + 1]
                sr = o.SR[t, :t + 1, 0, 0]
                gl = o.GLs[t, :t + 1, 0, 0]              # G^<(s, t)
                sl = -np.conj(o.SLs[t, :t + 1, 0, 0])    # Sigma^<(t, s)
                ga = np.conj(o.GR[t, :t + 1, 0, 0])      # G^A(s, t)
                acc += o.h * np.sum(wt * (sr * gl + sl * ga))
                acc += -1j * np.einsum("a,ab,b->", o.STV[t, :, 0, 0], o.Q, o.gvt(t)[:, 0, 0])
            out[t] = (-1j * acc / nk).real
        return out
