"""Pins of the oracle's equilibrium (Matsubara) Dyson solver on the DLR grid
(Eq. KBEM):
- the Bethe lattice converges to the semicircle G^M (closed form);
- a free Nambu level with pairing reproduces its closed-form G^M;
- the converged G^M solves the Dyson equation at Matsubara frequencies that
  were not used to determine it (second Born and Holstein terms included);
- the second-Born Matsubara bubble of a normal Nambu G equals the spin-basis
  -U^2 G_up(tau) G_dn(tau) G_dn(-tau);
- propagating the KBE from an interacting equilibrium with no drive keeps
  the state time-translation invariant: G^R(t, t') depends on t - t' only,
  which fails if any of the mixed self-energies or the Matsubara self-energy
  had the wrong sign or factor.
"""
import numpy as np
import pytest

import kbe_workloads as wk
from oracle.kbe import KBEOracle
from oracle.matsubara import MatsubaraOracle
from oracle.models import make_model

BETA = 5.0


@pytest.fixture(scope="module")
def mo():
    tau, om = wk.dlr_grid(100.0, 1e-12, BETA)
    return MatsubaraOracle(tau, om, BETA)


def test_bethe_semicircle(mo):
    G, _, it, err = mo.solve("bethe", np.array([[[0.3]]]), {"v": 1.0}, tol=1e-13, mix=0.7)
    assert np.abs(G[0, :, 0, 0] - wk.semicircle_gm(mo.tau, BETA, 0.3)).max() < 1e-10


def test_free_nambu_level(mo):
    em = np.array([[0.1, 0.3], [0.3, -0.1]])
    G, _, _, _ = mo.solve("nambu", em[None], {"v": 0.0}, tol=1e-13)
    assert np.abs(G[0] - wk.free_level_gm(mo.tau, BETA, em)).max() < 1e-9


@pytest.mark.parametrize("params", [{"v": 1.0, "U": 1.2}, {"v": 1.0, "g": 0.5, "w0": 0.6}])
def test_dyson_holds_off_the_nodes(mo, params):
    em = np.array([[0.2, 0.0], [0.0, -0.2]])
    G, e_eff, it, err = mo.solve("nambu", em[None], params, tol=1e-13, mix=0.6)
    assert err < 1e-12
    S = mo.sigma("nambu", G, params)[0]
    cg = np.linalg.solve(mo.Kt, -G[0].reshape(mo.r, -1))
    cs = np.linalg.solve(mo.Kt, -S.reshape(mo.r, -1))
    for n in (0, 3, 17, 60, 250):
        nu = (2 * n + 1) * np.pi / BETA
        kn = 1.0 / (1j * nu - mo.om)
        g = (kn @ cg).reshape(2, 2)
        s = (kn @ cs).reshape(2, 2)
        res = np.abs(g - np.linalg.inv(1j * nu * np.eye(2) - e_eff[0] - s)).max()
        assert res < 1e-9, (n, res)


def test_bubble_spin_basis(mo):
    r = mo.r
    gu = wk.semicircle_gm(mo.tau, BETA, 0.2).real    # two distinct Matsubara functions
    gd = wk.semicircle_gm(mo.tau, BETA, -0.1).real
    G = np.zeros((1, r, 2, 2), complex)
    G[0, :, 0, 0] = gu
    G[0, :, 1, 1] = -mo.xi * mo.reversed(gd)     # G22(tau) = -G_dn(-tau) = -xi G_dn(beta - tau)
    S = mo.sigma("nambu", G, {"v": 0.0, "U": 1.0})
    gd_minus = mo.xi * mo.reversed(gd)           # G_dn(-tau)
    assert np.allclose(S[0, :, 0, 0], -gu * gd * gd_minus, rtol=1e-9, atol=1e-10)


def test_interacting_equilibrium_is_stationary(mo):
    em = np.array([[0.15, 0.0], [0.0, -0.15]])
    params = {"v": 1.0, "U": 1.0, "g": 0.4, "w0": 0.8}
    G, e_eff, _, err = mo.solve("nambu", em[None], params, tol=1e-13, mix=0.6)
    nt, h, k = 50, 0.05, 5
    eps = np.broadcast_to(e_eff[0], (nt + 1, 2, 2)).astype(complex)
    A = np.zeros(nt + 1)
    U = np.full(nt + 1, params["U"])
    model = make_model("nambu", {"v": 1.0, "A": A, "U": U, "g": 0.4, "w0": 0.8})
    o = KBEOracle(nt, h, k, BETA, eps, G[0], mo.tau, mo.om, model, tol=1e-13)
    o.run()
    assert np.isfinite(o.GR).all() and np.isfinite(o.GLs).all()
    dev = 0.0
    for d in range(1, 30):
        vals = np.array([o.GR[t + d, t] for t in range(nt - d)])
        dev = max(dev, float(np.abs(vals - vals[0]).max()))
    assert dev < 1e-5, dev
    rho = np.array([o.rho(t) for t in range(nt)])
    assert np.abs(rho - rho[0]).max() < 1e-5


def test_lattice_interacting_equilibrium_is_stationary():
    """2D Hubbard 4 x 4 in second Born: the lattice Matsubara solution is a
    stationary state of the lockstep real-time oracle."""
    from oracle.lattice import LatticeOracle
    beta, L, U = 4.0, 4, 1.5
    tau, om = wk.dlr_grid(60.0, 1e-12, beta)
    mo = MatsubaraOracle(tau, om, beta)
    m = np.arange(L) * 2 * np.pi / L
    ek = (-2 * (np.cos(np.repeat(m, L)) + np.cos(np.tile(m, L))))
    G, _, _, err = mo.solve("lattice2b", ek[:, None, None].astype(complex), {"L": L, "U": U}, tol=1e-13, mix=0.6)
    assert err < 1e-12
    nt, h, k = 40, 0.05, 5
    eps = np.broadcast_to(ek[:, None, None, None], (L * L, nt + 1, 1, 1)).astype(complex)
    o = LatticeOracle(L, nt, h, k, beta, eps, G, tau, om, np.full(nt + 1, U), tol=1e-13).run()
    dev = 0.0
    for q in (0, 5):
        gr = o.orcs[q].GR[..., 0, 0]
        assert np.isfinite(gr).all() and np.isfinite(o.orcs[q].GLs).all()
        for d in range(1, 25):
            vals = np.array([gr[t + d, t] for t in range(nt - d)])
            dev = max(dev, float(np.abs(vals - vals[0]).max()))
    assert dev < 1e-4, dev          # h = 0.05 on a band of width 8


def test_paper_phases_of_the_attractive_hubbard_example():
    """The two states of the paper's driven-superconductor example (Sec. 4.1
    and its timing figure: U = 2 on the Bethe lattice, superconducting at
    beta = 18, disordered at beta = 1).  The Matsubara iteration with the
    symmetry-breaking pairing field 1e-4 for the first 5 iterations converges
    to a paired state at beta = 18: non-zero anomalous G^M and Fock pairing
    field.  At beta = 1 the pairing dies out and the normal state remains."""
    for beta, lam, paired in ((18.0, 100.0, True), (1.0, 40.0, False)):
        tau, om = wk.dlr_grid(lam, 1e-10, beta)
        mo = MatsubaraOracle(tau, om, beta)
        G, e, it, err = mo.solve("nambu", np.zeros((1, 2, 2)), {"v": 1.0, "U": 2.0}, tol=1e-12, mix=0.5,
                                 eta=1e-4, n_eta=5, max_iter=5000)
        assert err < 1e-12 and it > 5
        anom = np.abs(G[0, :, 0, 1]).max()
        if paired:
            assert anom > 0.1 and abs(e[0, 0, 1]) > 0.1, (anom, e[0, 0, 1])
        else:
            assert anom < 1e-10 and abs(e[0, 0, 1]) < 1e-10, (anom, e[0, 0, 1])


def test_superconducting_equilibrium_is_stationary():
    """Propagating the paper's superconducting equilibrium (U = 2, beta = 18,
    Bethe lattice, no drive) keeps it stationary: G^R(t + d, t) independent
    of t and rho constant, anomalous parts included, to the discretisation
    error (which falls at least 8-fold when h halves).  This fixes every
    anomalous term of the real-time functionals against the Matsubara ones:
    a flipped Fock sign, a missing sigma_z on the mixed hybridisation, or a
    wrong sign or factor of the mixed bubble leave deviations of 0.03 or more."""
    beta = 18.0
    tau, om = wk.dlr_grid(100.0, 1e-10, beta)
    mo = MatsubaraOracle(tau, om, beta)
    G, _, _, err = mo.solve("nambu", np.zeros((1, 2, 2)), {"v": 1.0, "U": 2.0}, tol=1e-13, mix=0.5, eta=1e-4,
                            n_eta=5, max_iter=5000)
    assert err < 1e-12 and np.abs(G[0, :, 0, 1]).max() > 0.1
    devs = []
    for nt, h in ((40, 0.05), (80, 0.025)):
        model = make_model("nambu", {"v": 1.0, "A": np.zeros(nt + 1), "U": np.full(nt + 1, 2.0)})
        o = KBEOracle(nt, h, 5, beta, np.zeros((nt + 1, 2, 2), complex), G[0], tau, om, model, tol=1e-13).run()
        dev = 0.0
        for d in range(1, nt // 2):
            vals = np.array([o.GR[t + d, t] for t in range(nt - d)])
            dev = max(dev, float(np.abs(vals - vals[0]).max()))
        rho = np.array([o.rho(t) for t in range(nt)])
        assert abs(rho[0][0, 1]) > 0.2                       # the pair amplitude is there
        devs.append(max(dev, float(np.abs(rho - rho[0]).max())))
    assert devs[1] < 2e-6 and devs[0] / devs[1] > 8, devs
