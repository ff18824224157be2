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
"""
from __future__ import annotations

import numpy as np


def _fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


class Model:
    name = "none"
    self_consistent = False

    def __init__(self, params=None):
        self.params = dict(params or {})

    def eval_step(self, st, T):
        st.SR[T, :T + 1] = 0.0
        st.SLs[T, :T + 1] = 0.0
        st.STV[T] = 0.0


class Bethe(Model):
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


def make_model(name, params=None):
    return {"none": Model, "bethe": Bethe, "bath": Bath}[name](params)
