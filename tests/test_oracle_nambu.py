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
  vector-potential pulse (the anomalous components stay zero);
- one site with a pairing field, by exact diagonalisation: Fock + bubble +
  exchange agree with it through U^2, the Holstein-Migdal term through g^2
  (the residual falls as U^3 and g^4); the Holstein term also against the
  independent-boson closed form at half filling.
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


def test_holstein_matches_independent_boson_model_to_order_g2():
    """v = U = 0 and eps = 0 (half filling): one site coupled to a free phonon
    through g (b + b^dagger)(n - 1), the independent-boson model.  Its exact
    Green's function (Lang-Firsov transformation) to order g^2, with
    lambda = g / w0:
        G^M(tau)  = -(1/2) [1 - lambda^2 ((2 n_B + 1) - (n_B + 1) e^{-w0 tau} - n_B e^{w0 tau})],
        G^R(t, 0) = -i [1 - lambda^2 (2 n_B + 1)(1 - cos w0 t)],
        G^<(t, 0) = (i/2) [1 - lambda^2 ((2 n_B + 1)(1 - cos w0 t) - i sin w0 t)]
    (the level shifts of the phonon-induced attraction cancel at this order at
    half filling).  The Migdal self-energy holds every order-g^2 diagram (the
    Hartree one vanishes at half filling), so the oracle's G^M and its real-time
    G started from it differ from these by O(g^4): the residual falls 16-fold
    when g halves.  A wrong factor, n_B or sign in D0 (greater, lesser or
    mixed branch) leaves an O(g^2) residual that falls only 4-fold."""
    from oracle.kbe import KBEOracle
    from oracle.matsubara import MatsubaraOracle
    from oracle.models import make_model
    w0, nt, h, k = 0.6, 80, 0.05, 5
    tau, om = wk.dlr_grid(100.0, 1e-12, BETA)
    mo = MatsubaraOracle(tau, om, BETA)
    nb = 1.0 / np.expm1(BETA * w0)
    t = np.arange(nt) * h
    res = []
    for g in (0.06, 0.03):
        lam2 = (g / w0) ** 2
        G, _, _, err = mo.solve("nambu", np.zeros((1, 2, 2)), {"v": 0.0, "g": g, "w0": w0}, tol=1e-14, mix=0.7)
        assert err < 1e-13
        gm = -0.5 * (1 - lam2 * ((2 * nb + 1) - (nb + 1) * np.exp(-w0 * tau) - nb * np.exp(w0 * tau)))
        gr = -1j * (1 - lam2 * (2 * nb + 1) * (1 - np.cos(w0 * t)))
        gl = 0.5j * (1 - lam2 * ((2 * nb + 1) * (1 - np.cos(w0 * t)) - 1j * np.sin(w0 * t)))
        model = make_model("nambu", {"v": 0.0, "g": g, "w0": w0, "A": np.zeros(nt + 1), "U": np.zeros(nt + 1)})
        o = KBEOracle(nt, h, k, BETA, np.zeros((nt + 1, 2, 2), complex), G[0], tau, om, model, tol=1e-13).run()
        r = []
        for c in (0, 1):
            corr = np.abs(gr - (-1j)).max()                # the order-g^2 term itself
            r.append(np.abs(G[0, :, c, c] - gm).max())
            r.append(np.abs(o.GR[:nt, 0, c, c] - gr).max())
            r.append(np.abs(-np.conj(o.GLs[:nt, 0, c, c]) - gl).max())   # G^<(t, 0) = -[G^<(0, t)]^*
            assert max(r[-3:]) < 0.03 * corr, (g, r[-3:], corr)
        assert np.abs(G[0, :, 0, 1]).max() == 0.0 and np.abs(o.GR[..., 0, 1]).max() < 1e-14
        res.append(np.array(r))
    ratio = res[0] / res[1]
    assert (ratio > 12).all() and (ratio < 20).all(), ratio


def test_holstein_paired_site_matches_exact_diagonalisation():
    """The same site with a pairing field delta (anomalous G): here the
    sigma_z sandwich of the Migdal term decides the sign of the anomalous
    self-energy.  Exact diagonalisation with a truncated phonon space is the
    truth; the Migdal G^M and real-time G differ from it by O(g^4) (every
    order-g^2 diagram is kept and the Hartree one vanishes at eps = 0), so the
    residual falls 16-fold when g halves.  At g = 0 the two agree to the
    discretisation error."""
    from oracle.kbe import KBEOracle
    from oracle.matsubara import MatsubaraOracle
    from oracle.models import make_model
    from _closed_forms import nambu_site
    w0, delta, nt, h, k = 0.6, 0.3, 80, 0.05, 5
    tau, om = wk.dlr_grid(100.0, 1e-12, BETA)
    mo = MatsubaraOracle(tau, om, BETA)
    em = np.array([[0.0, delta], [delta, 0.0]])
    t = np.arange(nt) * h
    res = []
    for g in (0.0, 0.06, 0.03):
        G, _, _, err = mo.solve("nambu", em[None], {"v": 0.0, "g": g, "w0": w0}, tol=1e-13, mix=0.7)
        assert err < 1e-12
        model = make_model("nambu", {"v": 0.0, "g": g, "w0": w0, "A": np.zeros(nt + 1), "U": np.zeros(nt + 1)})
        o = KBEOracle(nt, h, k, BETA, np.broadcast_to(em, (nt + 1, 2, 2)).astype(complex), G[0], tau, om, model,
                      tol=1e-13).run()
        gr, gl, gm = nambu_site(0.0, delta, BETA, t, tau, g=g, w0=w0)
        gl_o = -np.conj(np.swapaxes(o.GLs[:nt, 0], -1, -2))          # G^<(t, 0) = -[G^<(0, t)]^dagger
        res.append(np.array([np.abs(G[0] - gm).max(), np.abs(o.GR[:nt, 0] - gr).max(), np.abs(gl_o - gl).max()]))
    assert res[0].max() < 1e-9, res[0]
    corr = np.abs(nambu_site(0.0, delta, BETA, t, tau, g=0.06, w0=w0)[0] - nambu_site(0.0, delta, BETA, t, tau)[0]).max()
    assert res[1].max() < 0.03 * corr, (res[1], corr)
    ratio = res[1] / res[2]
    assert (ratio > 12).all() and (ratio < 20).all(), ratio


def test_second_born_paired_site_matches_exact_diagonalisation():
    """The attractive Hubbard term of Eq. Model on one site, -U (n_up - 1/2)(n_dn - 1/2),
    with a pairing field delta and no hybridisation: Fock (Eq. SigmaF) plus
    bubble and exchange (Eq. Sigma2B) hold every diagram through order U^2, so
    the self-consistent G^M and the real-time G started from it differ from
    exact diagonalisation by O(U^3): the residual falls about 8-fold when U
    halves.  A wrong Fock sign leaves an O(U) residual (2-fold), a dropped or
    sign-flipped exchange term with anomalous components an O(U^2) one
    (4-fold).  The model is given the external eps; it adds the Fock shift."""
    from oracle.kbe import KBEOracle
    from oracle.matsubara import MatsubaraOracle
    from oracle.models import make_model
    from _closed_forms import nambu_site
    delta, nt, h, k = 0.3, 80, 0.05, 5
    tau, om = wk.dlr_grid(100.0, 1e-12, BETA)
    mo = MatsubaraOracle(tau, om, BETA)
    em = np.array([[0.0, delta], [delta, 0.0]])
    t = np.arange(nt) * h
    res = []
    for U in (0.1, 0.05):
        G, e, _, err = mo.solve("nambu", em[None], {"v": 0.0, "U": U}, tol=1e-13, mix=0.7)
        assert err < 1e-12
        model = make_model("nambu", {"v": 0.0, "A": np.zeros(nt + 1), "U": np.full(nt + 1, U)})
        o = KBEOracle(nt, h, k, BETA, np.broadcast_to(em, (nt + 1, 2, 2)).astype(complex), G[0], tau, om, model,
                      tol=1e-13).run()
        gr, gl, gm = nambu_site(0.0, delta, BETA, t, tau, U=-U)
        gl_o = -np.conj(np.swapaxes(o.GLs[:nt, 0], -1, -2))          # G^<(t, 0) = -[G^<(0, t)]^dagger
        res.append(np.array([np.abs(G[0] - gm).max(), np.abs(o.GR[:nt, 0] - gr).max(), np.abs(gl_o - gl).max()]))
        if U == 0.1:
            corr = np.abs(gr - nambu_site(0.0, delta, BETA, t, tau)[0]).max()
            assert res[-1].max() < 0.02 * corr, (res[-1], corr)
    ratio = res[0] / res[1]
    assert (ratio > 6).all() and (ratio < 10).all(), ratio
