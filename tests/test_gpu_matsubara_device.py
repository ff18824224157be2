"""The equilibrium Dyson solve on the device (hkbe_solve_matsubara, Eq. KBEM)
against the oracle's Matsubara solver (oracle/matsubara.py) and the
library's host solver: Bethe, Nambu with U, Holstein and a pairing field
(the symmetry-broken state), and the 2D Hubbard lattice on the full and the
reflection-reduced k-set, up to C3's 16 x 16 grid; then a real-time
propagation from the installed G^M against the oracle."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import KBEOracle
from oracle.matsubara import MatsubaraOracle
from oracle.models import make_model

pytestmark = pytest.mark.gpu


def _handle(tau, om, beta, eps0, model, params, nt=20, nao=1):
    """A handle with the DLR grid, eps(t) = eps0 at every t and the model set."""
    n_inst = eps0.shape[0]
    st = pk.Stepper(nt, 0.02, 5, beta, nao=nao, n_inst=n_inst, tol=1e-13, max_iter=80)
    eps = np.broadcast_to(eps0[:, None], (n_inst, nt + 1, nao, nao)).astype(complex)
    st.set_inputs(tau, om, None, eps, model, params)
    return st


def test_bethe_matches_host_and_oracle():
    beta = 5.0
    tau, om = wk.dlr_grid(100.0, 1e-12, beta)
    eps0 = np.array([[[0.0]], [[0.3]], [[-0.45]]], complex)
    params = np.array([[1.0], [0.8], [1.2]])
    st = _handle(tau, om, beta, eps0, pk.MODEL_BETHE, params)
    G, it, err = pk.hkbe_solve_matsubara(st.h, 3, len(tau), 1, mix=0.5, tol=1e-13)
    Gh, _, ith, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_BETHE, eps0, params, mix=0.5, tol=1e-13)
    mo = MatsubaraOracle(tau, om, beta)
    for n in range(3):
        Go, _, _, _ = mo.solve("bethe", eps0[n:n + 1], {"v": params[n, 0]}, tol=1e-13, mix=0.5)
        assert np.abs(G[n] - Go[0]).max() < 1e-10
    assert np.abs(G - Gh).max() < 1e-11 and abs(it - ith) <= 1 and err < 1e-13
    st.close()


@pytest.mark.parametrize("beta,lam,e0,params,U,eta", [
    (5.0, 100.0, 0.15, [0.8], 0.7, 0.0),              # second Born
    (5.0, 100.0, 0.15, [1.0, 0.4, 0.8], 1.0, 0.0),    # second Born + Holstein
    (18.0, 100.0, 0.0, [1.0], 2.0, 1e-4)])            # the paper's superconducting point
def test_nambu_matches_oracle(beta, lam, e0, params, U, eta):
    """Nambu impurity of the Bethe lattice: second Born (U), optional
    Holstein (g, w0), and at beta = 18, U = 2 a pairing field for the first
    five iterations, which leaves the superconducting solution (anomalous
    G_01 != 0)."""
    tau, om = wk.dlr_grid(lam, 1e-12 if not eta else 1e-10, beta)
    em = np.array([[[e0, 0.0], [0.0, -e0]]], complex)
    kw = dict(U_eq=U, eta=eta, n_eta=5 if eta else 0, mix=0.5, tol=1e-12, max_iter=5000)
    st = _handle(tau, om, beta, em, pk.MODEL_NAMBU, np.array([params]), nao=2)
    G, it, _ = pk.hkbe_solve_matsubara(st.h, 1, len(tau), 2, **kw)
    pd = {"v": params[0], "U": U}
    if len(params) == 3:
        pd.update(g=params[1], w0=params[2])
    Go, _, _, _ = MatsubaraOracle(tau, om, beta).solve("nambu", em, pd, tol=1e-12, mix=0.5, eta=eta,
                                                       n_eta=kw["n_eta"], max_iter=5000)
    Gh, _, ith, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_NAMBU, em, [params], **kw)
    anom = np.abs(G[0, :, 0, 1]).max()
    print(f"Nambu U={U} eta={eta}: device {it} iterations, host {ith}; "
          f"max |G - G_oracle| {np.abs(G - Go).max():.2e}, anomalous {anom:.3f}")
    assert np.abs(G - Go).max() < 1e-10 and np.abs(G - Gh).max() < 1e-10
    assert (anom > 0.1) if eta else (anom < 1e-12)
    st.close()


@pytest.mark.parametrize("L,ysymm", [(4, False), (4, True), (16, False), (16, True)])
def test_lattice_matches_oracle(L, ysymm):
    """Half-filled 2D Hubbard lattice in second Born, U = 2, beta = 10 (C3's
    grid at L = 16): device solve on the full or reflection-reduced k-set
    against the oracle's full-grid solution at the same k-points."""
    beta, U = 10.0, 2.0
    tau, om = wk.dlr_grid(100.0, 1e-10, beta)
    m = np.arange(L) * 2 * np.pi / L
    ek = (-2 * (np.cos(np.repeat(m, L)) + np.cos(np.tile(m, L))))[:, None, None].astype(complex)
    kset = [x * L + y for x in range(L) for y in range(L // 2 + 1)] if ysymm else list(range(L * L))
    params = np.array([[float(L), 1.0] if ysymm else [float(L)]] * len(kset))
    st = _handle(tau, om, beta, ek[kset], pk.MODEL_LATTICE2B, params)
    G, it, _ = pk.hkbe_solve_matsubara(st.h, len(kset), len(tau), 1, U_eq=U, mix=0.5, tol=1e-12, max_iter=2000)
    Go, _, _, _ = MatsubaraOracle(tau, om, beta).solve("lattice2b", ek, {"L": L, "U": U}, tol=1e-12, mix=0.5,
                                                       max_iter=2000)
    print(f"lattice L={L} ysymm={ysymm}: {it} iterations, max |G - G_oracle| {np.abs(G - Go[kset]).max():.2e}")
    assert np.abs(G - Go[kset]).max() < 1e-10
    st.close()


def test_propagation_from_device_equilibrium():
    """Nambu with Holstein and U: G^M from the device solve, then a driven
    propagation; the oracle starts from its own G^M (from its own solver)."""
    beta, nt, h, k = 5.0, 60, 0.04, 5
    tau, om = wk.dlr_grid(100.0, 1e-12, beta)
    em = np.array([[0.15, 0.0], [0.0, -0.15]])
    par = [1.0, 0.4, 0.8]
    Go, e_eff, _, _ = MatsubaraOracle(tau, om, beta).solve("nambu", em[None], {"v": 1.0, "U": 1.0, "g": 0.4,
                                                                               "w0": 0.8}, tol=1e-13, mix=0.6)
    t = np.arange(nt) * h
    A = np.concatenate([[0.0], 0.4 * np.sin(1.2 * t) * np.exp(-(t - 1.5) ** 2 / 0.5)])
    Uv = np.full(nt + 1, 1.0)
    eps = np.broadcast_to(em, (nt + 1, 2, 2)).astype(complex)
    o = KBEOracle(nt, h, k, beta, eps, Go[0], tau, om,
                  make_model("nambu", {"v": 1.0, "A": A, "U": Uv, "g": 0.4, "w0": 0.8}), tol=1e-14)
    o.run()
    st = pk.Stepper(nt, h, k, beta, nao=2, tol=1e-13, max_iter=80)
    st.set_inputs(tau, om, None, eps[None], pk.MODEL_NAMBU, np.array([par]))
    G, _, _ = pk.hkbe_solve_matsubara(st.h, 1, len(tau), 2, U_eq=1.0, mix=0.6, tol=1e-13)
    assert np.abs(G - Go).max() < 1e-10
    pk.hkbe_set_drive(st.h, A[None], Uv[None])
    st.run()
    GR, GL, GTV = st.dense(0)
    idx = np.tril_indices(nt)
    ref = max(np.abs(o.GR[idx]).max(), np.abs(o.GLs[idx]).max(), np.abs(o.GTV).max())
    err = max(np.abs(GR[idx] - o.GR[idx]).max(), np.abs(GL[idx] - o.GLs[idx]).max(), np.abs(GTV - o.GTV).max())
    assert err / ref < 1e-10, err
    st.close()


def test_argument_errors():
    beta = 5.0
    tau, om = wk.dlr_grid(100.0, 1e-12, beta)
    st = _handle(tau, om, beta, np.array([[[0.2]]], complex), pk.MODEL_BETHE, np.array([[1.0]]))
    for kw in (dict(mix=0.0), dict(mix=1.5), dict(max_iter=0), dict(n_eta=-1), dict(tol=-1.0)):
        with pytest.raises(pk.HKBEError):
            pk.hkbe_solve_matsubara(st.h, 1, len(tau), 1, **kw)
    with pytest.raises(pk.HKBEError) as e:          # not converged in 2 iterations: the last iterate stays
        pk.hkbe_solve_matsubara(st.h, 1, len(tau), 1, tol=1e-15, max_iter=2)
    assert e.value.code == pk.HKBE_ERR_NOCONV
    pk.hkbe_solve_matsubara(st.h, 1, len(tau), 1, tol=1e-13)
    st.bootstrap()
    with pytest.raises(pk.HKBEError):               # after the bootstrap
        pk.hkbe_solve_matsubara(st.h, 1, len(tau), 1)
    st.close()
