"""Pins for the FP64 oracle stepper against closed forms, exact
diagonalisation and invariants (no GPU).

Every closed form lives in ``tests/_closed_forms.py`` and is written from the
definitions of Sec. 2.1, never from the discrete scheme.  Tolerances come from
the convergence order observed when h is halved (global error ~ h^k for the
order-k BDF/Gregory scheme of Appendix A).
"""
import numpy as np
import pytest

import kbe_workloads as wk
from oracle.kbe import KBEOracle, from_workload
from oracle.models import make_model

from _closed_forms import bethe, quadratic

BETA = 5.0
TAU, OM = wk.dlr_grid(100.0, 1e-12, BETA)
EPS2 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])


def _run_quadratic(eps_d, model, H_full, nt, h, k, rho_mode=0):
    no = eps_d.shape[0]
    eps = np.broadcast_to(eps_d, (nt + 1, no, no)).astype(complex)
    ts = np.arange(nt) * h
    GR, GL, GTV, GM = quadratic(H_full, BETA, ts, TAU, slice(0, no))
    o = KBEOracle(nt, h, k, BETA, eps, GM, TAU, OM, model, tol=1e-14, rho_mode=rho_mode)
    o.run()
    idx = np.tril_indices(nt)
    eR = np.abs(o.GR[idx] - GR[idx]).max()
    # GLs[T, t] = G^<(t, T)
    eL = np.abs(o.GLs[idx] - np.swapaxes(GL, 0, 1)[idx]).max()
    eT = np.abs(o.GTV - GTV).max()
    return max(eR, eL, eT), o


def test_sigma0_matrix_level_closed_form():
    """Sigma = 0 with a non-diagonal Hermitian 2x2 level (Sec. 3.3 G^HF forms)."""
    errs = []
    for nt, h in [(24, 0.1), (48, 0.05)]:
        e, o = _run_quadratic(EPS2, make_model("none"), EPS2, nt, h, k=4)
        errs.append(e)
    assert errs[1] < 1e-7
    assert errs[0] / errs[1] > 2 ** 3.5          # order-4 convergence


def _bath_setup():
    V = np.array([[0.5, 0.3j], [-0.2, 0.4]])
    eb = np.array([0.7, -0.9])
    H = np.block([[EPS2, V], [V.conj().T, np.diag(eb)]])
    return V, eb, H


@pytest.mark.parametrize("rho_mode", [0, 1])
def test_bath_matches_exact_diagonalisation(rho_mode):
    """Impurity (2 orbitals) coupled to 2 bath levels by a non-commuting V:
    G_dd from the 4x4 single-particle problem (pins operator ordering in every
    history integral, the mixed convolution and both rho schemes)."""
    V, eb, H = _bath_setup()
    model = make_model("bath", {"V": V, "eb": eb})
    errs = []
    for nt, h in [(32, 0.1), (64, 0.05)]:
        e, o = _run_quadratic(EPS2, model, H, nt, h, k=4, rho_mode=rho_mode)
        errs.append(e)
    assert errs[1] < 3e-6
    assert errs[0] / errs[1] > 2 ** 3.5


def test_bethe_j1_closed_form_and_order():
    errs = []
    for nt, h in [(40, 0.1), (80, 0.05)]:
        w = wk.c1_workload(seed=0, nt=nt, h=h, k=5, dlr_eps=1e-12)
        o = from_workload(w, tol=1e-14)
        o.run()
        e0 = w["eps"][0, 1, 0, 0].real
        GR, GL = bethe(np.full(nt, e0), h, nt, BETA, e0)
        idx = np.tril_indices(nt)
        eR = np.abs(o.GR[..., 0, 0][idx] - GR[idx]).max()
        eL = np.abs(o.GLs[..., 0, 0][idx] - GL.T[idx]).max()
        errs.append(max(eR, eL))
    assert errs[1] < 3e-7
    assert errs[0] / errs[1] > 2 ** 4.5          # order-5 convergence


def test_bethe_smooth_drive_order5():
    """Driven uniform level eps(t) = 0.3 sin(1.3 t): the level only multiplies
    G by the phase exp(-i int_{t'}^{t} eps) (gauge argument on the contour)."""
    errs = []
    for nt, h in [(40, 0.1), (80, 0.05)]:
        w = wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, dlr_eps=1e-12)
        n = np.arange(-1, nt)
        w["eps"][0, :, 0, 0] = 0.3 * np.sin(1.3 * np.maximum(n, 0) * h) * (n >= 0)
        w["gm"][0, :, 0, 0] = wk.semicircle_gm(w["tau"], BETA, 0.0)
        o = from_workload(w, tol=1e-14)
        o.run()
        ts = np.arange(nt) * h
        cum = 0.3 / 1.3 * (1 - np.cos(1.3 * ts))
        ph = np.exp(-1j * (cum[:, None] - cum[None, :]))
        GR, GL = bethe(np.zeros(nt), h, nt, BETA, 0.0)
        idx = np.tril_indices(nt)
        errs.append(max(np.abs(o.GR[..., 0, 0][idx] - (GR * ph)[idx]).max(),
                        np.abs(o.GLs[..., 0, 0][idx] - (GL * ph).T[idx]).max()))
    assert errs[1] < 3e-6
    assert errs[0] / errs[1] > 2 ** 4.5


def test_bethe_level_quench_first_order():
    """Level quench eps0: 0 -> 1 at t = 1 (the C2 protocol, moved earlier).
    The jump sits on a grid point, so the scheme is first order there: the
    error against the exact phase exp(-i max(t-1, 0) + i max(t'-1, 0)) halves
    with h."""
    errs = []
    for nt, h in [(40, 0.1), (80, 0.05)]:
        w = wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, quench=(0.0, 1.0, 1.0), dlr_eps=1e-12)
        o = from_workload(w, tol=1e-14)
        o.run()
        ts = np.arange(nt) * h
        cum = np.maximum(ts - 1.0, 0.0)
        ph = np.exp(-1j * (cum[:, None] - cum[None, :]))
        GR, GL = bethe(np.zeros(nt), h, nt, BETA, 0.0)
        idx = np.tril_indices(nt)
        errs.append(max(np.abs(o.GR[..., 0, 0][idx] - (GR * ph)[idx]).max(),
                        np.abs(o.GLs[..., 0, 0][idx] - (GL * ph).T[idx]).max()))
    assert errs[1] < 2.5 * 0.05
    assert 1.8 < errs[0] / errs[1] < 2.2


def test_invariants_bethe():
    nt, h = 64, 0.05
    runs = []
    for beta in (5.0, 1.0):
        w = wk.bethe_workload(nt=nt, h=h, k=5, beta=beta, seed=3, dlr_eps=1e-12)
        o = from_workload(w, tol=1e-14)
        o.run()
        runs.append(o)
    o = runs[0]
    g = o.GR[..., 0, 0]
    assert np.allclose(np.diag(g), -1j, atol=1e-15)
    # Sigma^R = v^2 G^R depends on G^R alone and G^R(t,t) = -i: the retarded
    # component cannot depend on the thermal state (beta, G^M, G^<, G^tv).
    assert np.abs(runs[0].GR - runs[1].GR).max() < 1e-13
    assert np.abs(runs[0].GLs - runs[1].GLs).max() > 1e-2
    # undriven: time-translation invariance up to the discretisation error
    for s in range(0, 30):
        d = np.array([g[T, T - s] for T in range(s, nt)])
        assert np.abs(d - d[0]).max() < 5e-7
    n = (-1j * np.array([o.GLs[t, t, 0, 0] for t in range(nt)])).real
    assert n.max() - n.min() < 1e-6            # particle number conserved


def test_rho_diagonal_preserves_hermiticity():
    """The diagonal rho equation (Sec. 3.3) maps Hermitian data to a Hermitian
    rho: the anti-Hermitian part seeded by the bootstrap square must not grow."""
    V, eb, H = _bath_setup()
    model = make_model("bath", {"V": V, "eb": eb})
    e, o = _run_quadratic(EPS2, model, H, 64, 0.05, k=4, rho_mode=1)
    ah = [np.abs(o.rho(t) - o.rho(t).conj().T).max() for t in range(64)]
    assert max(ah[5:]) <= 2.0 * max(ah[:5]) + 1e-15


# ---- planted mistakes: each pin must catch a plausible bug -----------------

def _patched_error(monkeypatch, patch):
    V, eb, H = _bath_setup()
    model = make_model("bath", {"V": V, "eb": eb})
    with monkeypatch.context() as m:
        patch(m)
        e, _ = _run_quadratic(EPS2, model, H, 32, 0.1, k=4)
    return e


def test_pin_catches_dropped_convolution(monkeypatch):
    e = _patched_error(monkeypatch, lambda m: m.setattr(
        KBEOracle, "conv", lambda self, t: 0 * np.einsum("axy,aiyz->ixz", self.STV[t], self.Wconv)))
    assert e > 1e-3


def test_pin_catches_transposed_history_product(monkeypatch):
    orig = KBEOracle.sR_x

    def swapped(self, a, b):
        return orig(self, a, b).T
    e = _patched_error(monkeypatch, lambda m: m.setattr(KBEOracle, "sR_x", swapped))
    assert e > 1e-3


def test_pin_catches_wrong_gregory_weight(monkeypatch):
    from oracle import weights as W
    orig = W.Weights.rule

    def bad(self, n):
        w = orig(self, n).copy()
        if n >= 2 * self.k + 1:
            w[1] += 0.01
        return w
    e = _patched_error(monkeypatch, lambda m: m.setattr(W.Weights, "rule", bad))
    assert e > 1e-4


def _bethe_energy(o, T, W):
    """n(T) = -i G^<(T,T) and E_kin(T) = -i [Sigma * G]^<(T,T) (Langreth rule
    for the lesser component of the contour convolution at equal times,
    Sec. 2.1): h sum_l w_l [Sigma^R(T,l) G^<(l,T) + Sigma^<(T,l) G^A(l,T)]
    - i int Sigma^tv(T,tau) G^vt(tau,T) dtau, with the Gregory rule of step T
    and the DLR quadrature (Sec. 2.5)."""
    h = o.h
    wt = W.rule(T)
    GA = np.conj(np.swapaxes(o.GR[T, :T + 1], -1, -2))
    SLT = np.array([(-np.conj(o.SLs[T, l].T) if l < T else o.SLs[T, T]) for l in range(T + 1)])
    conv = h * np.einsum("l,lxy,lyz->xz", wt, o.SR[T, :T + 1], o.GLs[T, :T + 1])
    conv += h * np.einsum("l,lxy,lyz->xz", wt, SLT, GA)
    v = np.einsum("ab,bxy->axy", o.Q, o.gvt(T))
    conv += -1j * np.einsum("axy,ayz->xz", o.STV[T], v)
    return (-1j * o.GLs[T, T])[0, 0].real, (-1j * conv)[0, 0]


def test_bethe_energy_conserved_at_order_k():
    """Undriven Bethe lattice from its equilibrium: the energy per site,
    E = eps0 n + E_kin with E_kin = -i [Sigma * G]^<(t,t), stays at its
    closed form int w A(w) f(w) dw (A the semicircle of half-bandwidth 2
    centred on eps0; eps0 n is then int eps0 A f) at every step, and its
    drift falls as h^k (k = 5) when h halves."""
    from oracle.weights import Weights
    W = Weights(5)
    drift, dev = [], []
    for nt, h in [(40, 0.1), (80, 0.05)]:
        w = wk.c1_workload(seed=0, nt=nt, h=h, k=5, dlr_eps=1e-12)
        o = from_workload(w, tol=1e-14)
        o.run()
        e0 = w["eps"][0, 1, 0, 0].real
        # closed forms by Gauss-Chebyshev quadrature of the second kind
        th = np.arange(1, 4001) * np.pi / 4001
        om = e0 + 2 * np.cos(th)
        wq = (2 / np.pi) * np.pi / 4001 * np.sin(th) ** 2
        f = 0.5 * (1 - np.tanh(0.5 * BETA * om))
        n_cl, ek_cl = np.sum(wq * f), np.sum(wq * f * (om - e0))
        E = np.array([[e0 * n + ek.real, ek.imag] for n, ek in (_bethe_energy(o, T, W) for T in range(6, nt))])
        assert np.abs(E[:, 1]).max() < 1e-12                      # E_kin is real
        drift.append(np.abs(E[:, 0] - E[0, 0]).max())
        dev.append(np.abs(E[:, 0] - (e0 * n_cl + ek_cl)).max())
    assert dev[1] < 1e-6
    assert drift[1] < 1e-6 and drift[0] / drift[1] > 2 ** 4     # order k = 5 (measured 2^4.7)
