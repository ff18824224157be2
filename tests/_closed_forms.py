"""Closed-form Green's functions used to pin the oracle (written from the
definitions in Sec. 2.1 / Table 1, by exact diagonalisation or special
functions; nothing here touches the discrete scheme)."""
import numpy as np
from scipy.special import j1


def _fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


def quadratic(H, beta, ts, taus, sel, xi=-1):
    """Non-interacting system with single-particle Hamiltonian H; returns the
    `sel` block of G^R(t,t'), G^<(t,t'), G^tv(t,tau), G^M(tau) on the grids."""
    E, U = np.linalg.eigh(H)
    f = _fermi(E, beta)
    Us = U[sel, :]
    d = ts[:, None] - ts[None, :]
    ph = np.exp(-1j * E[None, None, :] * d[:, :, None])
    GR = -1j * np.einsum("xa,tsa,ya->tsxy", Us, ph, Us.conj())
    GL = 1j * np.einsum("xa,tsa,a,ya->tsxy", Us, ph, f, Us.conj())
    tv = np.exp(-1j * E[None, None, :] * ts[:, None, None]) * np.exp(E[None, None, :] * taus[None, :, None])
    GTV = -xi * 1j * np.einsum("xa,tia,a,ya->tixy", Us, tv, f, Us.conj())
    GM = -np.einsum("xa,ia,a,ya->ixy", Us, np.exp(-E[None, :] * taus[:, None]), 1 - f, Us.conj())
    return GR, GL, GTV, GM


def bethe(eps_of_t, h, nt, beta, eps_eq, v=1.0, nquad=4000):
    """Bethe lattice (semicircle of half-bandwidth 2v) with a time-dependent
    uniform level eps(t) (the level only multiplies by a phase):
    G^R(t,t') = -i e^{-i int eps} J1(2v(t-t'))/(v(t-t')),
    G^<(t,t') = i e^{-i int eps} int A(w) f(w) e^{-i (w - eps_eq)(t - t')} dw."""
    ts = np.arange(nt) * h
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (eps_of_t[1:] + eps_of_t[:-1]) * h)])
    phase = np.exp(-1j * (cum[:, None] - cum[None, :]))
    d = ts[:, None] - ts[None, :]
    dd = np.where(np.abs(d) > 0, d, 1.0)
    jr = np.where(np.abs(d) > 0, j1(2 * v * dd) / (v * dd), 1.0)
    GR = -1j * phase * jr
    j = np.arange(1, nquad + 1)
    th = j * np.pi / (nquad + 1)
    x = np.cos(th)
    wq = np.pi / (nquad + 1) * np.sin(th) ** 2 * (2 / np.pi)
    xx = 2 * v * x
    f = _fermi(eps_eq + xx, beta)
    GL = 1j * phase * np.einsum("q,q,tsq->ts", wq, f, np.exp(-1j * xx[None, None, :] * d[:, :, None]))
    return GR, GL
