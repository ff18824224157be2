"""Pins of the oracle's Nambu model (driven hybridisation of Eq. Hybrid,
second-Born bubble and exchange of Eq. Sigma2B, Fock term of Eq. SigmaF).

- U = 0, no drive, normal state: the two Nambu components are independent
  Bethe lattices with levels +eps0 and -eps0 (closed form J1 / semicircle);
- the bubble for a normal (diagonal) Nambu G equals the textbook spin-basis
  second-order self-energy U^2 G_up^> G_dn^> G_dn^<(t', t), mapped through
  psi = (d_up, d_dn^dagger);
- the Sigma2B index pattern is covariant under the U(1) gauge transformation
  psi -> exp(i theta sigma_z) psi (a transposed or misplaced bar breaks it);
- a normal initial state stays normal under an interaction quench and a
  vector-potential pulse (the anomalous components stay zero).
"""
import numpy as np
import pytest

import kbe_workloads as wk
from oracle.kbe import from_workload
from oracle.models import _bar_products
from _closed_forms import bethe

BETA = 5.0


def test_nambu_u0_reduces_to_two_bethe_lattices():
    errs = []
    for nt, h in [(40, 0.1), (80, 0.05)]:
        e0 = 0.3
        w = wk.nambu_workload(nt=nt, h=h, k=5, beta=BETA, v=1.0, eps0=e0, dlr_eps=1e-12)
        o = from_workload(w, tol=1e-14)
        o.run()
        idx = np.tril_indices(nt)
        e = 0.0
        for c, lev in ((0, e0), (1, -e0)):
            GR, GL = bethe(np.full(nt, lev), h, nt, BETA, lev)
            e = max(e, np.abs(o.GR[..., c, c][idx] - GR[idx]).max(), np.abs(o.GLs[..., c, c][idx] - GL.T[idx]).max())
        assert np.abs(o.GR[..., 0, 1]).max() < 1e-13 and np.abs(o.GLs[..., 1, 0]).max() < 1e-13
        errs.append(e)
    assert errs[1] < 3e-6                         # the hole component has the larger constant
    assert errs[0] / errs[1] > 2 ** 4.5           # order-5 convergence


def test_bubble_matches_spin_basis_second_order():
    rng = np.random.default_rng(3)
    n = 7
    def rnd():
        return rng.normal(size=n) + 1j * rng.normal(size=n)
    gup_g, gdn_g, gdn_l_rev, gdn_l, gdn_g_rev = rnd(), rnd(), rnd(), rnd(), rnd()
    # Nambu psi = (d_up, d_dn^dagger):  G22^>(t,t') = -G_dn^<(t',t),  G22^<(t',t) = -G_dn^>(t,t')
    X = np.zeros((n, 2, 2), complex)
    Y = np.zeros((n, 2, 2), complex)
    X[:, 0, 0] = gup_g                 # G11^>(t,t') = G_up^>(t,t')
    X[:, 1, 1] = -gdn_l_rev            # G22^>(t,t') = -G_dn^<(t',t)
    Y[:, 1, 1] = -gdn_g                # G22^<(t',t) = -G_dn^>(t,t')
    Y[:, 0, 0] = rnd()
    S = _bar_products(X, Y)
    spin = gup_g * gdn_g * gdn_l_rev   # U^2 G_up^>(t,t') G_dn^>(t,t') G_dn^<(t',t), U = 1
    assert np.allclose(S[:, 0, 0], spin, rtol=1e-14, atol=1e-14)
    assert np.abs(S[:, 0, 1]).max() == 0 and np.abs(S[:, 1, 0]).max() == 0


def test_sigma2b_gauge_covariance():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(9, 2, 2)) + 1j * rng.normal(size=(9, 2, 2))
    Y = rng.normal(size=(9, 2, 2)) + 1j * rng.normal(size=(9, 2, 2))
    s = np.array([1.0, -1.0])
    for th in (0.3, 1.1, -2.0):
        g = np.exp(1j * th * (s[:, None] - s[None, :]))    # G_ij -> e^{i th (s_i - s_j)} G_ij, both orders
        lhs = _bar_products(X * g, Y * g)
        assert np.allclose(lhs, _bar_products(X, Y) * g, rtol=1e-13, atol=1e-13)
    # a transposed reversed-time factor is caught
    bad = np.zeros_like(X)
    for i in range(2):
        for j in range(2):
            bad[..., i, j] = X[..., i, j] * X[..., 1 - i, 1 - j] * Y[..., 1 - i, 1 - j]
    g = np.exp(1j * 0.7 * (s[:, None] - s[None, :]))
    bad2 = np.zeros_like(X)
    for i in range(2):
        for j in range(2):
            bad2[..., i, j] = (X * g)[..., i, j] * (X * g)[..., 1 - i, 1 - j] * (Y * g)[..., 1 - i, 1 - j]
    assert not np.allclose(bad2, bad * g)


@pytest.mark.parametrize("rho_mode", [0, 1])
def test_normal_state_stays_normal_under_quench_and_pulse(rho_mode):
    nt, h = 60, 0.05
    w = wk.nambu_workload(nt=nt, h=h, k=4, beta=BETA, v=1.0, eps0=0.2, U=1.0, t_quench=0.5,
                          A0=0.4, Omega=1.3, tc=1.5, width=0.5, rho_mode=rho_mode)
    o = from_workload(w, tol=1e-13)
    o.run()
    assert np.abs(o.GR[..., 0, 1]).max() < 1e-13 and np.abs(o.GLs[..., 0, 1]).max() < 1e-13
    assert np.abs(o.GTV[..., 1, 0]).max() < 1e-13
    # the interaction and the pulse act: the normal components moved off the U = 0 result
    w0 = wk.nambu_workload(nt=nt, h=h, k=4, beta=BETA, v=1.0, eps0=0.2, rho_mode=rho_mode)
    o0 = from_workload(w0, tol=1e-13)
    o0.run()
    assert np.abs(o.GLs[-1, :, 0, 0] - o0.GLs[-1, :, 0, 0]).max() > 1e-3
    rho = np.array([o.rho(t) for t in range(nt)])
    # the horizontal scheme keeps rho Hermitian to the discretisation error; the
    # diagonal one does not grow the anti-Hermitian part left by the start square
    ah = np.abs(rho - np.conj(np.swapaxes(rho, -1, -2))).max(axis=(1, 2))
    if rho_mode == 0:
        assert ah.max() < 1e-4, ah.max()
    else:
        assert ah[5:].max() <= ah[:5].max() + 1e-12, (ah[:5].max(), ah[5:].max())


def test_fock_term_enters_eps_with_pairing():
    """Free Nambu level with a pairing term (v = 0) and an interaction quench:
    the anomalous density is nonzero, so the Fock term shifts the off-diagonal
    level by -U rho_12."""
    nt, h = 40, 0.05
    w = wk.nambu_workload(nt=nt, h=h, k=4, beta=BETA, v=0.0, eps0=0.1, pairing=0.3, U=0.8, t_quench=0.2)
    o = from_workload(w, tol=1e-13)
    o.run()
    T = nt - 1
    rho = o.rho(T)
    assert abs(rho[0, 1]) > 1e-2
    assert np.allclose(o.eps[T + 1][0, 1], 0.3 - 0.8 * rho[0, 1], atol=1e-12)
    assert np.allclose(o.eps[T + 1][0, 0], 0.1, atol=1e-15)


def test_holstein_term_g0_limit_and_effect():
    """g = 0 reproduces the plain model bit for bit; g = 0.5 changes it."""
    kw = dict(nt=40, h=0.05, k=4, beta=BETA, v=1.0, eps0=0.1, A0=0.3, Omega=1.0, tc=1.0, width=0.5)
    a = from_workload(wk.nambu_workload(**kw), tol=1e-13).run()
    w0 = wk.nambu_workload(**kw)
    w0["wl"].params.update({"g": 0.0, "w0": 0.6})
    b = from_workload(w0, tol=1e-13).run()
    assert np.array_equal(a.GR, b.GR) and np.array_equal(a.GLs, b.GLs)
    c = from_workload(wk.nambu_workload(g=0.5, w0=0.6, **kw), tol=1e-13).run()
    assert np.abs(c.GLs[-1, :, 0, 0] - a.GLs[-1, :, 0, 0]).max() > 1e-3
