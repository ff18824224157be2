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



def nambu_site(eps, delta, beta, ts, taus, U=0.0, g=0.0, w0=1.0, nph=16):
    """One site with level eps, pairing field delta, a Hubbard term and a
    Holstein phonon,
        H = eps (n - 1) + delta (c_up^+ c_dn^+ + c_dn c_up) + U (n_up - 1/2)(n_dn - 1/2)
            + w0 b^+ b + g (b + b^+)(n - 1),
    solved by exact diagonalisation in the Fock space of the two spins times
    nph phonon states (one state when g = 0).  With the Nambu spinor
    psi = (c_up, c_dn^+) it returns G^R(t, 0), G^<(t, 0) on ts and G^M(tau)
    on taus, each (len, 2, 2):
        G^>_ij(t) = -i <psi_i(t) psi_j^+>,  G^<_ij(t) = i <psi_j^+ psi_i(t)>,
        G^M_ij(tau) = -<psi_i(tau) psi_j^+>  (0 < tau < beta)."""
    if g == 0.0:
        nph = 1
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    cu = np.kron(a, np.eye(2))
    cd = np.kron(np.diag([1.0, -1.0]), a)          # Jordan-Wigner sign
    nu, nd = cu.T @ cu, cd.T @ cd
    n1 = nu + nd - np.eye(4)
    He = eps * n1 + delta * (cu.T @ cd.T + cd @ cu) + U * (nu - 0.5 * np.eye(4)) @ (nd - 0.5 * np.eye(4))
    b = np.diag(np.sqrt(np.arange(1.0, nph)), 1)
    H = np.kron(He, np.eye(nph)) + w0 * np.kron(np.eye(4), b.T @ b) + g * np.kron(n1, b + b.T)
    E, V = np.linalg.eigh(H)
    E = E - E.min()
    P = [V.T @ np.kron(cu, np.eye(nph)) @ V, V.T @ np.kron(cd.T, np.eye(nph)) @ V]
    w = np.exp(-beta * E)
    w = w / w.sum()
    def corr(wgt, ph):                             # sum_mn wgt_mn ph_mn P_i[m,n] P_j[m,n]^*
        return np.array([[np.sum(wgt * ph * P[i] * P[j].conj()) for j in range(2)] for i in range(2)])
    dE = E[:, None] - E[None, :]
    GR, GL = [], []
    for t in ts:
        ph = np.exp(1j * t * dE)
        gg = -1j * corr(w[:, None], ph)
        gl = 1j * corr(w[None, :], ph)
        GR.append(gg - gl)
        GL.append(gl)
    Z = np.exp(-beta * E).sum()
    GM = [-corr(np.exp(-(beta - s) * E[:, None] - s * E[None, :]) / Z, 1.0).real for s in taus]
    return np.array(GR), np.array(GL), np.array(GM)


def hubbard_cluster(L, U, beta, ts, taus):
    """The L x L periodic Hubbard cluster (L = 2: 8 spin orbitals, 256 states),
        H = -sum_<ij>,s c_is^+ c_js + U sum_i (n_i,up - 1/2)(n_i,dn - 1/2),
    the hopping summed over the four neighbour directions with wrap-around,
    solved by exact diagonalisation.  Returns, per k = 2 pi (m_x, m_y) / L
    (index m_x L + m_y) and for spin up, G^R_k(t, 0), G^<_k(t, 0) on ts and
    G^M_k(tau) on taus, with c_k = N^{-1/2} sum_i e^{-i k.r_i} c_i."""
    ns = L * L
    nm = 2 * ns                                    # mode 2 i + s: site i, spin s
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    z = np.diag([1.0, -1.0])
    c = []
    for m in range(nm):                            # Jordan-Wigner
        op = np.ones((1, 1))
        for q in range(nm):
            op = np.kron(op, z if q < m else (a if q == m else np.eye(2)))
        c.append(op)
    xy = [(i // L, i % L) for i in range(ns)]
    dim = 2 ** nm
    H = np.zeros((dim, dim))
    for i, (x, y) in enumerate(xy):
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            j = ((x + dx) % L) * L + (y + dy) % L
            for s in range(2):
                H -= c[2 * i + s].T @ c[2 * j + s]
    for i in range(ns):
        H += U * (c[2 * i].T @ c[2 * i] - 0.5 * np.eye(dim)) @ (c[2 * i + 1].T @ c[2 * i + 1] - 0.5 * np.eye(dim))
    E, V = np.linalg.eigh(H)
    E = E - E.min()
    w = np.exp(-beta * E)
    Z = w.sum()
    dE = E[:, None] - E[None, :]
    GR = np.zeros((ns, len(ts)), complex)
    GL = np.zeros((ns, len(ts)), complex)
    GM = np.zeros((ns, len(taus)))
    for q in range(ns):
        kx, ky = 2 * np.pi * np.array(xy[q]) / L
        ck = sum(np.exp(-1j * (kx * x + ky * y)) * c[2 * i] for i, (x, y) in enumerate(xy)) / np.sqrt(ns)
        A = np.abs(V.T @ ck @ V) ** 2              # |<m| c_k |n>|^2
        for n, t in enumerate(ts):
            ph = np.exp(1j * t * dE)
            gl = 1j * np.sum(w[None, :] * ph * A) / Z
            GR[q, n] = -1j * np.sum(w[:, None] * ph * A) / Z - gl
            GL[q, n] = gl
        for n, s in enumerate(taus):
            GM[q, n] = -np.sum(np.exp(-(beta - s) * E[:, None] - s * E[None, :]) * A) / Z
    return GR, GL, GM
