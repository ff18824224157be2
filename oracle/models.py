"""Oracle: self-energy functionals evaluated at one time step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each model fills, for the time step T, the current retarded row
Sigma^R(T, t'), t' <= T, the current lesser column Sigma^<(t, T), t <= T (stored
as row T of the lower-triangular lesser storage, Sec. 2.1), and the mixed row
Sigma^tv(T, tau_i) on the DLR nodes.

  none   Sigma = 0
  bethe  Bethe lattice DMFT hybridisation Sigma = v^2 G (the single-orbital,
         undriven case of Eq. Hybrid, where t0-bar reduces to v)
  bath   bath levels eps_b coupled by the matrix V (Sigma = V g_b V^dagger, a
         fixed functional of time): g_b^R(t,t') = -i e^{-i eps_b (t-t')},
         g_b^<(t,t') = i n_b e^{-i eps_b (t-t')},
         g_b^tv(t, tau) = -xi i n_b e^{-i eps_b t} e^{eps_b tau}
         with n_b the Fermi occupation at beta (Sec. 3.3 forms of G^HF).
  nambu  driven Nambu DMFT: hybridisation (Eq. Hybrid) + second Born (Eq.
         Sigma2B) + Fock (Eq. SigmaF), see Nambu
"""
from __future__ import annotations

import numpy as np


def _fermi(e, beta):
    """Fermi function 1/(e^{beta e} + 1) (Sec. 2.1), overflow-safe."""
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


class Model:
    """Sigma = 0 (free propagation); base of the self-energy functionals that
    fill Sigma^R(T, .), Sigma^<(., T) and Sigma^tv(T, .) of step T (Sec. 3.4)."""
    name = "none"
    self_consistent = False

    def __init__(self, params=None):
        self.params = dict(params or {})

    def eval_step(self, st, T):
        st.SR[T, :T + 1] = 0.0
        st.SLs[T, :T + 1] = 0.0
        st.STV[T] = 0.0


class Bethe(Model):
    """Bethe-lattice DMFT hybridisation Sigma = v^2 G (Eq. Hybrid, Sec. 3.1)."""
    name = "bethe"
    self_consistent = True

    def eval_step(self, st, T):
        v2 = self.params.get("v", 1.0) ** 2
        st.SR[T, :T + 1] = v2 * st.GR[T, :T + 1]
        st.SLs[T, :T + 1] = v2 * st.GLs[T, :T + 1]
        st.STV[T] = v2 * st.GTV[T]


class Bath(Model):
    """Bath levels eps_b (N_b) coupled through the N_o x N_b matrix V:
    Sigma^X(t, t') = V g_b^X(t, t') V^dagger with g_b diagonal."""
    name = "bath"

    def eval_step(self, st, T):
        V = np.atleast_2d(np.asarray(self.params["V"], dtype=complex))
        eb = np.atleast_1d(np.asarray(self.params["eb"], dtype=float))
        nb = _fermi(eb, st.beta)
        h = st.h
        tp = np.arange(T + 1)

        def dress(g):        # g: (..., N_b) diagonal entries -> V diag(g) V^dag
            return np.einsum("xb,...b,yb->...xy", V, g, V.conj())
        st.SR[T, :T + 1] = dress(-1j * np.exp(-1j * np.outer(T - tp, eb) * h))
        # Sigma^<(t, T) for t <= T: V diag(i n_b e^{-i eb (t - T)}) V^dag
        st.SLs[T, :T + 1] = dress(1j * nb * np.exp(-1j * np.outer(tp - T, eb) * h))
        st.STV[T] = dress((-st.xi) * 1j * nb * np.exp(-1j * eb * T * h)
                          * np.exp(np.outer(st.tau, eb)))


def _bar_products(X, Y):
    """Eq. Sigma2B index pattern for 2 x 2 Nambu matrices (bar i = 1 - i):
    out_ij = X_ij X_{bi bj} Y_{bj bi} - X_{bi j} X_{i bj} Y_{bj bi},
    for stacks X[..., 2, 2] (the two equal-time-order factors) and Y (the
    reversed-time factor)."""
    out = np.zeros_like(X)
    for i in range(2):
        for j in range(2):
            bi, bj = 1 - i, 1 - j
            out[..., i, j] = (X[..., i, j] * X[..., bi, bj] - X[..., bi, j] * X[..., i, bj]) * Y[..., bj, bi]
    return out


class Nambu(Model):
    """Nambu (2 x 2) impurity of a Bethe-lattice DMFT with the driven
    hybridisation of Eq. Hybrid, the second-Born bubble and exchange diagrams
    of Eq. Sigma2B and the Fock term of Eq. SigmaF (Sec. 4.1).

    params: v   hopping scale (Delta carries v^2; the paper's case is v = 1)
            A   vector potential, array [nt+1]: A[0] on the equilibrium branch,
                A[t+1] at time t (Peierls phases t0-bar = diag(e^{iA}, e^{-iA}))
            U   interaction, array [nt+1], same indexing (U(t) U(t') in Eq.
                Sigma2B; the equilibrium-branch value enters the mixed part)

    With s = (1, -1) the hybridisation of Eq. Hybrid is, element by element,
        Delta_ij(t, t') = v^2 s_i s_j G_ij(t, t') cos(s_i A(t) - s_j A(t')).
    The bubble and exchange give Sigma^>(T, t) from G^>(T, t) and G^<(t, T),
    Sigma^<(T, t) from G^<(T, t) and G^>(t, T); Sigma^R = Sigma^> - Sigma^< on
    t <= T.  The mixed part uses G^tv(T, tau) and G^vt(tau, T) the same way
    (the imaginary branch is latest on the contour).  The Fock term
    Sigma^F_ij(t) = -U(t) rho_ij(t) [i = bar j] is time-local: it is added to
    the external eps(t) every time Sigma is evaluated.

    Optional Holstein coupling (params g, w0; the C4 configuration): the
    unrenormalised Migdal self-energy Sigma^≷(t,t') = i g^2 D0^≷(t,t')
    sigma_z G^≷(t,t') sigma_z with the free phonon propagator
    D0^>(t,t') = -i[(n_B+1) e^{-i w0 (t-t')} + n_B e^{i w0 (t-t')}],
    D0^<(t,t') = D0^>(t',t), n_B = 1/(e^{beta w0} - 1), and on the mixed
    branch D0^tv(t,tau) = -i[(n_B+1) e^{i w0 t - w0 tau} + n_B e^{-i w0 t + w0 tau}].
    The paper names this approximation but prints no formula for it.  Pinned
    against the independent-boson model (half filling, closed form to order
    g^2) and against exact diagonalisation of a site with a pairing field:
    both agree with Migdal through order g^2."""
    name = "nambu"
    self_consistent = True

    def eval_step(self, st, T):
        if not hasattr(self, "eps_ext"):
            self.eps_ext = st.eps.copy()
        v2 = float(self.params.get("v", 1.0)) ** 2
        A = np.asarray(self.params.get("A", np.zeros(st.nt + 1)), dtype=float)
        U = np.asarray(self.params.get("U", np.zeros(st.nt + 1)), dtype=float)
        s = np.array([1.0, -1.0])
        ss = np.outer(s, s)

        def dag(x):
            return np.conj(np.swapaxes(x, -1, -2))
        GR = st.GR[T, :T + 1]                     # G^R(T, t)
        GLc = st.GLs[T, :T + 1]                   # G^<(t, T)
        GLr = -dag(GLc)                           # G^<(T, t)
        GGr = GR + GLr                            # G^>(T, t)
        GGc = -dag(GGr)                           # G^>(t, T)
        uu = (U[T + 1] * U[1:T + 2])[:, None, None]
        Sg = uu * _bar_products(GGr, GLc)         # Sigma^>(T, t)
        Sl = uu * _bar_products(GLr, GGc)         # Sigma^<(T, t)
        ph = np.cos(s[None, :, None] * A[T + 1] - s[None, None, :] * A[1:T + 2][:, None, None])
        st.SR[T, :T + 1] = Sg - Sl + v2 * ss * GR * ph
        st.SLs[T, :T + 1] = -dag(Sl + v2 * ss * GLr * ph)
        Gtv = st.GTV[T]                           # G^tv(T, tau_i)
        Gvt = st.gvt(T)                           # G^vt(tau_i, T)
        ph0 = np.cos(s[:, None] * A[T + 1] - s[None, :] * A[0])
        st.STV[T] = U[T + 1] * U[0] * _bar_products(Gtv, Gvt) + v2 * ss * Gtv * ph0
        g = float(self.params.get("g", 0.0))
        if g != 0.0:
            w0 = float(self.params["w0"])
            nb = 1.0 / np.expm1(st.beta * w0)
            dt = (T - np.arange(T + 1)) * st.h                  # t_T - t
            dg = -1j * ((nb + 1) * np.exp(-1j * w0 * dt) + nb * np.exp(1j * w0 * dt))   # D0^>(T, t)
            dl = -1j * ((nb + 1) * np.exp(1j * w0 * dt) + nb * np.exp(-1j * w0 * dt))   # D0^<(T, t)
            sg = 1j * g * g * dg[:, None, None] * ss * GGr
            sl = 1j * g * g * dl[:, None, None] * ss * GLr
            st.SR[T, :T + 1] += sg - sl
            st.SLs[T, :T + 1] += -dag(sl)
            tT = T * st.h
            dtv = -1j * ((nb + 1) * np.exp(1j * w0 * tT - w0 * st.tau) + nb * np.exp(-1j * w0 * tT + w0 * st.tau))
            st.STV[T] += 1j * g * g * dtv[:, None, None] * ss * Gtv
        rho = st.rho(T)
        sf = np.zeros((2, 2), complex)
        sf[0, 1] = -U[T + 1] * rho[0, 1]
        sf[1, 0] = -U[T + 1] * rho[1, 0]
        st.eps[T + 1] = self.eps_ext[T + 1] + sf


def make_model(name, params=None):
    """Self-energy functional by name: none, bethe, bath, nambu."""
    return {"none": Model, "bethe": Bethe, "bath": Bath, "nambu": Nambu}[name](params)
